// libtrees: the TREES epoch step on one B300 (sm_103a), behind the C ABI of
// include/trees.h.
//
// Three schedulers drive the same Phase-2 tile code (trees_programs.cuh):
//  - persistent: one cooperative launch.  Every block keeps its own copy of
//    the epoch-range stack (the join stack + NDRange stack of Sec. 5.2) in
//    shared memory and applies Phase 3 (Sec. 5.2.4) and Phase 1 (Sec. 5.2.2)
//    itself from the same global counters, so an epoch costs one grid
//    barrier (two when maps were scheduled).
//  - graph: a CUDA graph whose conditional WHILE node runs the epoch
//    kernel, the map kernel and a one-thread Phase-3 kernel per epoch.
//  - hostloop: the paper's own arrangement (Sec. 5.2.2-5.2.4): the host pops
//    the stacks, launches one kernel over the NDRange, reads nextFreeCore /
//    joinScheduled / mapScheduled back, and launches the map kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "trees.h"
#include "trees_impl/trees_dev.cuh"
#include "trees_impl/trees_programs.cuh"
#include "trees_batch.cuh"
#include "trees_impl/trees_kernels.cuh"

#include <chrono>
#include <deque>
#include <map>
#include <thread>

using namespace trees;

namespace {


// ------------------------------------------------------------------ kernels

// Zeroes the control block and the run's per-block statistics and writes the
// root task into TV entry 0 for epoch 0 (Sec. 5.2.1).
constexpr int SETUP_BLOCKS = 32;  // k_setup's grid: the statistics' clearing spread over a few SMs
__global__ void k_setup(Ctl *ctl, Conf c, uint32_t type, uint32_t a0, uint32_t a1, unsigned long long *blk) {
    // every block clears its share of the per-block statistics; block 0 sets up the control block and the root
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < (uint32_t)NBLK_STATS * 4u; i += gridDim.x * blockDim.x)
        blk[i] = 0ull;
    if (blockIdx.x != 0) return;
    unsigned int *w = reinterpret_cast<unsigned int *>(ctl);
    for (uint32_t i = threadIdx.x; i < sizeof(Ctl) / 4; i += blockDim.x) w[i] = 0u;
    __syncthreads();
    if (threadIdx.x == 0) {
        c.code[0] = enc(0u, type);
        c.a0[0] = a0;
        c.a1[0] = a1;
        c.link[0] = 0u;
        c.result[0] = 0ull;
        ctl->g_cen = 0u;
        ctl->g_lo = 0u;
        ctl->g_hi = 1u;
        ctl->g_base = 1u;
        ctl->g_next = 1u;
        ctl->g_e = 0u;
        ctl->g_sp = 0u;
        ctl->g_stop = 0u;
        ctl->peak = 1u;
        ctl->t_start = globaltimer();
    }
}

// BFS start: every level unknown but the source's, and the visited bits
// likewise.
__global__ void k_bfs_init(int32_t *level, uint32_t *visited, int32_t nv, int32_t src) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x)
        level[v] = (v == src) ? 0 : -1;
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < ((int64_t)nv + 31) / 32;
         w += (int64_t)gridDim.x * blockDim.x)
        visited[w] = w == src / 32 ? 1u << (src % 32) : 0u;
}

// SSSP start: every distance unknown but the source's; no vertex forked yet
// (the root task relaxes the source in epoch 0).
__global__ void k_sssp_init(unsigned long long *dist, uint32_t *sched, unsigned long long *used, int32_t nv,
                            int32_t src) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x) {
        dist[v] = (v == src) ? 0ull : ~0ull;
        sched[v] = 0u;
        used[v] = 0ull;  // never relaxed
    }
}

// Phase 2 of one epoch as its own kernel (graph and host-loop schedulers).
// from_ctl = 1: the epoch comes from the control block (graph); 0: from the
// arguments (host loop, grid sized to the NDRange as in Sec. 5.1.1).
template <int BS, int TPT>
__global__ void __launch_bounds__(BS) k_epoch(Ctl *ctl, Conf c, unsigned long long *blk, int from_ctl, uint32_t a_cen,
                                              uint32_t a_lo, uint32_t a_hi, uint32_t a_base, uint32_t a_e) {
    __shared__ Smem<BS> sm;
    if (threadIdx.x == 0) {
        sm.stop = vload(&ctl->err) != 0 || (from_ctl && vload(&ctl->g_stop) != 0u);
        if (from_ctl) {
            sm.cen = vload(&ctl->g_cen);
            sm.lo = vload(&ctl->g_lo);
            sm.hi = vload(&ctl->g_hi);
            sm.base = vload(&ctl->g_base);
            sm.next = vload(&ctl->g_e);
        } else {
            sm.cen = a_cen;
            sm.lo = a_lo;
            sm.hi = a_hi;
            sm.base = a_base;
            sm.next = a_e;
        }
    }
    __syncthreads();
    if (sm.stop) return;
    const uint32_t cen = sm.cen, lo = sm.lo, hi = sm.hi, base = sm.base, e = sm.next, ep = e % 3u;
    if (blockIdx.x == 0 && threadIdx.x == 0) clear_epoch_slot(ctl, (e + 1u) % 3u);
    Acc acc = {0u, 0u, 0u};
    int par = 0;
    bool jn = false;
    for (unsigned long long t0 = (unsigned long long)lo + (unsigned long long)blockIdx.x * (BS * TPT); t0 < hi;
         t0 += (unsigned long long)gridDim.x * (BS * TPT)) {
        TileLoad<TPT> L;
        tile_load<BS, TPT, PM_ALL>(c, t0, hi, LOAD_ON_DEMAND, L);
        jn |= epoch_tile<BS, TPT, PM_ALL>(c, ctl, sm, t0, hi, cen, base, ep, e, acc, par, LOAD_ON_DEMAND, L,
                                          hi - lo <= (uint32_t)(BS * TPT), 0u).joined;
        par ^= 1;
    }
    publish_join(ctl, ep, jn);
    trace_valid_add<BS>(c, e, acc.valid, sm);
    block_add_stats<BS>(blk, acc, sm);
}

// The map operations scheduled in one epoch, as their own kernel.
template <int BS>
__global__ void __launch_bounds__(BS) k_map(Ctl *ctl, Conf c, int from_ctl, uint32_t a_cen, uint32_t a_base,
                                            uint32_t a_e) {
    __shared__ Smem<BS> sm;
    if (threadIdx.x == 0) {
        sm.stop = vload(&ctl->err) != 0 || (from_ctl && vload(&ctl->g_stop) != 0u);
        sm.cen = from_ctl ? vload(&ctl->g_cen) : a_cen;
        sm.base = from_ctl ? vload(&ctl->g_base) : a_base;
        sm.next = from_ctl ? vload(&ctl->g_e) : a_e;
    }
    __syncthreads();
    if (sm.stop) return;
    const uint32_t cen = sm.cen, base = sm.base, e = sm.next, ep = e % 3u;
    const unsigned long long mt = vload(&ctl->mt_ctr[ep]), me = vload(&ctl->me_ctr[ep]);
    if (!(mt | me)) return;
    map_phase<BS, PM_ALL>(c, ctl, sm, ep, e, cen, base, mt, me);
}

// The partition sub-phase of one epoch's merges, as its own kernel.
template <int BS>
__global__ void __launch_bounds__(BS) k_partition(Ctl *ctl, Conf c, int from_ctl, uint32_t a_e) {
    if (vload(&ctl->err) != 0 || (from_ctl && vload(&ctl->g_stop) != 0u)) return;
    const uint32_t e = from_ctl ? vload(&ctl->g_e) : a_e, ep = e % 3u;
    const unsigned long long mt = vload(&ctl->mt_ctr[ep]);
    if (!needs_partition(mt)) return;
    partition_phase<BS>(c, mt, nullptr, 0u);
}

// Phase 3 + Phase 1 of the graph scheduler (one thread): updates the
// device-resident stacks and ends the WHILE loop when they are empty.
__global__ void k_phase3(Ctl *ctl, Conf c, cudaGraphConditionalHandle h) {
    if (threadIdx.x != 0) return;
    uint32_t cont = 1u;
    if (ctl->g_stop) {
        cont = 0u;
    } else {
        const uint32_t e = ctl->g_e, ep = e % 3u;
        const uint32_t cen = ctl->g_cen, lo = ctl->g_lo, hi = ctl->g_hi, base = ctl->g_base;
        const uint32_t f = *fork_ctr(ctl, ep), jf = ctl->join[ep];
        const unsigned long long mt = ctl->mt_ctr[ep], me = ctl->me_ctr[ep];
        uint32_t sp = ctl->g_sp, next = base;
        int ok = 1;
        if (jf) {
            if (sp < c.gstack_cap) c.gstack[sp++] = Range{cen, lo, hi, 1u};
            else ok = 0;
        }
        if (f) {
            if (sp < c.gstack_cap) c.gstack[sp++] = Range{cen + 1u, base, base + f, 0u};
            else ok = 0;
            next = base + f;
        } else if (!jf) {
            next = lo;
        }
        ctl->forks += f;
        ctl->peak = max(ctl->peak, base + f);
        if (c.trace_on && e < c.trace_cap) {
            trees_epoch_t r;
            r.cen = cen;
            r.lo = lo;
            r.hi = hi;
            r.valid = 0u;
            r.forks = f;
            r.joined = jf;
            r.maps = (uint32_t)(mt >> 40) + (uint32_t)(me >> 40);
            r.ns_phase2 = 0u;
            r.ns_partition = 0u;
            r.ns_map = 0u;
            r.t_ns = globaltimer();
            c.trace[e] = r;
        }
        const uint32_t ne = e + 1u;
        ctl->g_e = ne;
        ctl->g_next = next;
        if (!ok) set_err(ctl, TREES_ERR_STACK, e);
        if (ctl->err || !ok) {
            cont = 0u;
        } else if (sp == 0u) {
            cont = 0u;
        } else if (ne >= c.max_epochs) {
            set_err(ctl, TREES_ERR_EPOCH_LIMIT, ne);
            cont = 0u;
        } else {
            const Range r = c.gstack[--sp];
            ctl->g_cen = r.cen;
            ctl->g_lo = r.lo;
            ctl->g_hi = r.hi;
            ctl->g_base = next;
        }
        ctl->g_sp = sp;
        if (!cont) {
            ctl->g_stop = 1u;
            ctl->epochs = ne;
            ctl->final_next = next;
            ctl->t_end = globaltimer();
        }
    }
    if (ctl->err && !ctl->g_stop) {
        ctl->g_stop = 1u;
        ctl->epochs = ctl->g_e;
        ctl->t_end = globaltimer();
        cont = 0u;
    }
    cudaGraphSetConditional(h, cont);
}

// The critical-path floor: only grid barriers, same grid as k_persistent.
template <int BS>
__global__ void __launch_bounds__(BS) k_floor(Ctl *ctl, uint32_t iters, unsigned long long timeout_ns) {
    __shared__ Smem<BS> sm;
    uint32_t bar = 0;
    for (uint32_t i = 0; i < iters; ++i)
        if (!grid_sync<BS>(ctl, &bar, timeout_ns, sm)) break;
}

// ------------------------------------------------------------------ host side

struct Kern {
    const void *persistent, *epoch, *map, *floor, *partition;
};

template <int BS, int TPT>
Kern kern_for() {
    return Kern{nullptr, (const void *)k_epoch<BS, TPT>, (const void *)k_map<BS>, (const void *)k_floor<BS>,
                (const void *)k_partition<BS>};
}

// The persistent kernel compiled for a program.
const void *persistent_kernel(int program, int bs, int tpt) {
    switch (program) {
    case TREES_PROG_FIB: return persistent_kernel_fib(bs, tpt);
    case TREES_PROG_MERGESORT: return persistent_kernel_ms(bs, tpt);
    case TREES_PROG_NQUEENS: return persistent_kernel_nq(bs, tpt);
    case TREES_PROG_BFS: return persistent_kernel_bfs(bs, tpt);
    case TREES_PROG_SSSP: return persistent_kernel_sssp(bs, tpt);
    case TREES_PROG_FFT: return persistent_kernel_fft(bs, tpt);
    default: return persistent_kernel_trav(bs, tpt);
    }
}

bool kern_by(int bs, int tpt, Kern *k) {
    switch (bs * 10 + tpt) {
    case 1281: *k = kern_for<128, 1>(); return true;
    case 1282: *k = kern_for<128, 2>(); return true;
    case 1284: *k = kern_for<128, 4>(); return true;
    case 2561: *k = kern_for<256, 1>(); return true;
    case 2562: *k = kern_for<256, 2>(); return true;
    case 2564: *k = kern_for<256, 4>(); return true;
    case 5121: *k = kern_for<512, 1>(); return true;
    case 5122: *k = kern_for<512, 2>(); return true;
    case 5124: *k = kern_for<512, 4>(); return true;
    case 10241: *k = kern_for<1024, 1>(); return true;
    case 10242: *k = kern_for<1024, 2>(); return true;
    case 10244: *k = kern_for<1024, 4>(); return true;
    default: return false;
    }
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

constexpr int NMT = 7;  // tiled-map descriptor columns: kind, a, b, c, job, first tile, split
constexpr int NME = 5;  // element-map columns: first adjacency index, first element, job, tile's first descriptor, vertex

struct Layout {
    size_t off_dev, off_code, off_a0, off_a1, off_link, off_result;
    size_t off_mt[NMT], off_me[NME], off_trace, off_tvalid, off_gstack, off_blk, total;
};

Layout make_layout(size_t cap, size_t mcap, size_t trace_cap, size_t gstack_cap) {
    Layout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t r = o;
        o = align_up(o + bytes, 256);
        return r;
    };
    L.off_dev = take(sizeof(Dev));
    L.off_code = take(cap * 4);
    L.off_a0 = take(cap * 4);
    L.off_a1 = take(cap * 4);
    L.off_link = take(cap * 4);
    L.off_result = take(cap * 8);
    for (int i = 0; i < NMT; ++i) L.off_mt[i] = take(mcap * 4);
    for (int i = 0; i < NME; ++i) L.off_me[i] = take(mcap * 4);
    L.off_trace = take(trace_cap * sizeof(trees_epoch_t));
    L.off_tvalid = take(trace_cap * 4);
    L.off_gstack = take(gstack_cap * sizeof(Range));
    L.off_blk = take((size_t)NBLK_STATS * 4 * 8);
    L.total = o;
    return L;
}

void normalize(trees_config_t *c) {
    if (c->block_size == 0) c->block_size = 512;
    if (c->max_epochs == 0) c->max_epochs = 1u << 20;
    if (c->trace_cap == 0) c->trace_cap = 65536;
    if (c->timeout_ns == 0) c->timeout_ns = 2000000000ull;
    if (c->tasks_per_thread == 0) c->tasks_per_thread = 2;
}

}  // namespace

struct trees_ctx {
    int device = 0, sms = 0;
    trees_config_t cfg{};
    char *mem = nullptr;
    size_t bytes = 0;
    bool owns = false;
    Layout L{};
    Ctl *ctl = nullptr;
    Conf conf{};
    unsigned long long *blk = nullptr;
    uint32_t cap = 0, mcap = 0;
    int grid = 0, bs = 0;
    Kern kern{};
    cudaStream_t last_stream = nullptr;
    int last_grid = 0;               // grid of the last persistent run
    std::map<const void *, int> grid_cache;
    uint32_t *own_scratch = nullptr;
    size_t own_scratch_n = 0;
    unsigned long long *own_used = nullptr;  // SSSP relax records (one word per vertex)
    size_t own_used_n = 0;
    uint32_t *own_smp = nullptr;  // mergesort splitter samples (n/64 + 1 keys)
    size_t own_smp_n = 0;
    // graph scheduler
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaGraphNode_t gnode_epoch = nullptr, gnode_map = nullptr, gnode_p3 = nullptr, gnode_part = nullptr;
    cudaGraphConditionalHandle gh = 0;
    // host-loop scheduler
    std::vector<trees_epoch_t> host_trace;
    int last_sched = TREES_SCHED_PERSISTENT;
    int host_status = TREES_OK;
    Ctl *pinned_ctl = nullptr;
    // trees_sync's copies of the last run's status and root result (slot 0), in pinned host memory
    struct SyncPin {
        int err;
        int pad;
        unsigned long long res0;
    } *pin_sync = nullptr;
    bool res0_valid = false;  // pin_sync->res0 is slot 0's result of the last run
    bool res0_in_ctl = false;  // the last run's kernel left slot 0's result in ctl->res0 (beside err)
    // batched runs
    Job *d_jobs = nullptr;
    uint32_t *d_joff = nullptr;
    BatchDone *d_done = nullptr;
    BatchCtl *d_bc = nullptr;
    Job *h_jobs = nullptr;
    int32_t batch_cap = 0, batch_n = 0;
};

extern "C" {

void trees_default_config(trees_config_t *cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->block_size = 512;
    cfg->blocks_per_sm = 0;
    cfg->scheduler = TREES_SCHED_PERSISTENT;
    cfg->trace = 0;
    cfg->max_epochs = 1u << 20;
    cfg->trace_cap = 65536;
    cfg->timeout_ns = 2000000000ull;
    cfg->map_capacity = 0;
    cfg->inject_stall_epoch = -1;
    cfg->grid_blocks = 0;
    cfg->tasks_per_thread = 2;
}

static size_t bytes_for_cfg(size_t cap, const trees_config_t &c) {
    const size_t mcap = c.map_capacity ? (size_t)c.map_capacity : cap;
    return make_layout(cap, mcap, c.trace_cap, STK_CAP).total;
}

size_t trees_bytes_for(size_t capacity_slots, const trees_config_t *cfg) {
    trees_config_t c;
    if (cfg) c = *cfg;
    else trees_default_config(&c);
    normalize(&c);
    if (capacity_slots == 0 || capacity_slots > 0xFFFFFFFFull) return 0;
    return bytes_for_cfg(capacity_slots, c);
}

static int finish_create(trees_ctx *x) {
    if (cudaGetDevice(&x->device) != cudaSuccess) return TREES_ERR_CUDA;
    if (cudaDeviceGetAttribute(&x->sms, cudaDevAttrMultiProcessorCount, x->device) != cudaSuccess)
        return TREES_ERR_CUDA;
    if (!kern_by(x->cfg.block_size, x->cfg.tasks_per_thread, &x->kern)) return TREES_ERR_INVALID_ARG;
    x->bs = x->cfg.block_size;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, x->kern.epoch, x->bs, 0) != cudaSuccess || occ < 1)
        return TREES_ERR_CUDA;
    int per_sm = x->cfg.blocks_per_sm > 0 ? std::min(x->cfg.blocks_per_sm, occ) : occ;
    x->grid = x->sms * per_sm;
    if (x->cfg.grid_blocks > 0) x->grid = std::min(x->cfg.grid_blocks, x->sms * occ);
    char *m = x->mem;
    const Layout &L = x->L;
    x->ctl = reinterpret_cast<Ctl *>(m + L.off_dev);
    Conf &c = x->conf;
    std::memset(&c, 0, sizeof(c));
    c.code = reinterpret_cast<uint32_t *>(m + L.off_code);
    c.a0 = reinterpret_cast<uint32_t *>(m + L.off_a0);
    c.a1 = reinterpret_cast<uint32_t *>(m + L.off_a1);
    c.link = reinterpret_cast<uint32_t *>(m + L.off_link);
    c.result = reinterpret_cast<unsigned long long *>(m + L.off_result);
    c.cap = x->cap;
    uint32_t **mt[NMT] = {&c.mt_kind, &c.mt_a, &c.mt_b, &c.mt_c, &c.mt_job, &c.mt_tilebase, &c.mt_split};
    for (int i = 0; i < NMT; ++i) *mt[i] = reinterpret_cast<uint32_t *>(m + L.off_mt[i]);
    uint32_t **me[NME] = {&c.me_v, &c.me_base, &c.me_job, &c.me_tfd, &c.me_src};
    for (int i = 0; i < NME; ++i) *me[i] = reinterpret_cast<uint32_t *>(m + L.off_me[i]);
    c.mcap = x->mcap;
    c.trace = reinterpret_cast<trees_epoch_t *>(m + L.off_trace);
    c.trace_valid = reinterpret_cast<uint32_t *>(m + L.off_tvalid);
    c.trace_cap = x->cfg.trace_cap;
    c.trace_on = x->cfg.trace;
    c.max_epochs = x->cfg.max_epochs;
    c.stall_epoch = x->cfg.inject_stall_epoch;
    c.timeout_ns = x->cfg.timeout_ns;
    c.gstack = reinterpret_cast<Range *>(m + L.off_gstack);
    c.gstack_cap = STK_CAP;
    x->blk = reinterpret_cast<unsigned long long *>(m + L.off_blk);
    if (cudaMallocHost(&x->pinned_ctl, sizeof(Ctl)) != cudaSuccess) return TREES_ERR_CUDA;
    if (cudaMallocHost(&x->pin_sync, sizeof(trees_ctx::SyncPin)) != cudaSuccess) return TREES_ERR_CUDA;
    if (cudaMemset(x->ctl, 0, sizeof(Ctl)) != cudaSuccess) return TREES_ERR_CUDA;
    return TREES_OK;
}

// Co-resident grid for a kernel launched with `smem` bytes of dynamic shared
// memory, under the context's limits (cached).  Raises the kernel's dynamic
// shared memory limit on this device first when smem needs it.
static int kernel_grid(trees_ctx *x, const void *kern, size_t smem = 0) {
    if (!kern) return 0;
    auto it = x->grid_cache.find(kern);
    if (it != x->grid_cache.end()) return it->second;
    if (smem && cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, x->bs, smem) != cudaSuccess || occ < 1) return 0;
    const int per_sm = x->cfg.blocks_per_sm > 0 ? std::min(x->cfg.blocks_per_sm, occ) : occ;
    int g = x->sms * per_sm;
    if (x->cfg.grid_blocks > 0) g = std::min(x->cfg.grid_blocks, x->sms * occ);
    x->grid_cache[kern] = g;
    return g;
}

static int validate_cfg(const trees_config_t *cfg, trees_config_t *out) {
    if (cfg) *out = *cfg;
    else trees_default_config(out);
    normalize(out);
    if (out->block_size != 128 && out->block_size != 256 && out->block_size != 512 && out->block_size != 1024)
        return TREES_ERR_INVALID_ARG;
    if (out->scheduler < TREES_SCHED_PERSISTENT || out->scheduler > TREES_SCHED_HOSTLOOP) return TREES_ERR_INVALID_ARG;
    if (out->blocks_per_sm < 0 || out->grid_blocks < 0) return TREES_ERR_INVALID_ARG;
    if (out->tasks_per_thread != 1 && out->tasks_per_thread != 2 && out->tasks_per_thread != 4)
        return TREES_ERR_INVALID_ARG;
    return TREES_OK;
}

int trees_create(size_t capacity_slots, const trees_config_t *cfg, trees_ctx **out) {
    if (!out || capacity_slots == 0 || capacity_slots > 0xFFFFFFFFull) return TREES_ERR_INVALID_ARG;
    *out = nullptr;
    trees_ctx *x = new (std::nothrow) trees_ctx();
    if (!x) return TREES_ERR_INVALID_ARG;
    int rc = validate_cfg(cfg, &x->cfg);
    if (rc) {
        delete x;
        return rc;
    }
    x->cap = (uint32_t)capacity_slots;
    const uint64_t mc = x->cfg.map_capacity ? x->cfg.map_capacity : capacity_slots;
    if (mc > 0xFFFFFFFFull) {
        delete x;
        return TREES_ERR_INVALID_ARG;
    }
    x->mcap = (uint32_t)mc;
    x->L = make_layout(x->cap, x->mcap, x->cfg.trace_cap, STK_CAP);
    if (cudaMalloc(&x->mem, x->L.total) != cudaSuccess) {
        cudaGetLastError();
        delete x;
        return TREES_ERR_CUDA;
    }
    x->owns = true;
    x->bytes = x->L.total;
    rc = finish_create(x);
    if (rc) {
        trees_destroy(x);
        return rc;
    }
    *out = x;
    return TREES_OK;
}

int trees_create_on(void *dev_buf, size_t bytes, const trees_config_t *cfg, trees_ctx **out) {
    if (!out || !dev_buf || ((uintptr_t)dev_buf & 255u)) return TREES_ERR_INVALID_ARG;
    *out = nullptr;
    trees_ctx *x = new (std::nothrow) trees_ctx();
    if (!x) return TREES_ERR_INVALID_ARG;
    int rc = validate_cfg(cfg, &x->cfg);
    if (rc) {
        delete x;
        return rc;
    }
    // the largest capacity whose layout fits (binary search on slots)
    size_t lo = 0, hi = 0xFFFFFFFFull;
    while (lo < hi) {
        const size_t mid = lo + (hi - lo + 1) / 2;
        if (bytes_for_cfg(mid, x->cfg) <= bytes) lo = mid;
        else hi = mid - 1;
    }
    if (lo == 0) {
        delete x;
        return TREES_ERR_INVALID_ARG;
    }
    x->cap = (uint32_t)lo;
    x->mcap = x->cfg.map_capacity ? (uint32_t)std::min<uint64_t>(x->cfg.map_capacity, 0xFFFFFFFFull) : x->cap;
    x->L = make_layout(x->cap, x->mcap, x->cfg.trace_cap, STK_CAP);
    x->mem = static_cast<char *>(dev_buf);
    x->owns = false;
    x->bytes = bytes;
    rc = finish_create(x);
    if (rc) {
        trees_destroy(x);
        return rc;
    }
    *out = x;
    return TREES_OK;
}

void trees_destroy(trees_ctx *x) {
    if (!x) return;
    if (x->gexec) cudaGraphExecDestroy(x->gexec);
    if (x->graph) cudaGraphDestroy(x->graph);
    if (x->own_scratch) cudaFree(x->own_scratch);
    if (x->own_used) cudaFree(x->own_used);
    if (x->own_smp) cudaFree(x->own_smp);
    if (x->pinned_ctl) cudaFreeHost(x->pinned_ctl);
    if (x->pin_sync) cudaFreeHost(x->pin_sync);
    if (x->d_jobs) cudaFree(x->d_jobs);
    if (x->d_joff) cudaFree(x->d_joff);
    if (x->d_done) cudaFree(x->d_done);
    if (x->d_bc) cudaFree(x->d_bc);
    if (x->h_jobs) cudaFreeHost(x->h_jobs);
    if (x->owns && x->mem) cudaFree(x->mem);
    delete x;
}

size_t trees_capacity(const trees_ctx *x) { return x ? x->cap : 0; }

int trees_geometry(const trees_ctx *x, int32_t *grid_blocks, int32_t *block_size, int32_t *sms) {
    if (!x) return TREES_ERR_INVALID_ARG;
    if (grid_blocks) *grid_blocks = x->grid;
    if (block_size) *block_size = x->bs;
    if (sms) *sms = x->sms;
    return TREES_OK;
}

// Builds the graph of the graph scheduler once per context: a conditional
// WHILE node whose body is epoch kernel -> map kernel -> Phase-3 kernel.
static int build_graph(trees_ctx *x) {
    if (x->gexec) return TREES_OK;
    if (cudaGraphCreate(&x->graph, 0) != cudaSuccess) return TREES_ERR_CUDA;
    if (cudaGraphConditionalHandleCreate(&x->gh, x->graph, 1, cudaGraphCondAssignDefault) != cudaSuccess)
        return TREES_ERR_CUDA;
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = x->gh;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode;
    if (cudaGraphAddNode(&cnode, x->graph, nullptr, nullptr, 0, &cp) != cudaSuccess) return TREES_ERR_CUDA;
    cudaGraph_t body = cp.conditional.phGraph_out[0];

    static int from_ctl = 1;
    static uint32_t zero = 0;
    void *ep_args[] = {&x->ctl, &x->conf, &x->blk, &from_ctl, &zero, &zero, &zero, &zero, &zero};
    cudaKernelNodeParams kp;
    std::memset(&kp, 0, sizeof(kp));
    kp.func = const_cast<void *>(x->kern.epoch);
    kp.gridDim = dim3(x->grid);
    kp.blockDim = dim3(x->bs);
    kp.kernelParams = ep_args;
    if (cudaGraphAddKernelNode(&x->gnode_epoch, body, nullptr, 0, &kp) != cudaSuccess) return TREES_ERR_CUDA;
    void *part_args[] = {&x->ctl, &x->conf, &from_ctl, &zero};
    kp.func = const_cast<void *>(x->kern.partition);
    kp.kernelParams = part_args;
    if (cudaGraphAddKernelNode(&x->gnode_part, body, &x->gnode_epoch, 1, &kp) != cudaSuccess) return TREES_ERR_CUDA;
    void *map_args[] = {&x->ctl, &x->conf, &from_ctl, &zero, &zero, &zero};
    kp.func = const_cast<void *>(x->kern.map);
    kp.kernelParams = map_args;
    if (cudaGraphAddKernelNode(&x->gnode_map, body, &x->gnode_part, 1, &kp) != cudaSuccess) return TREES_ERR_CUDA;
    void *p3_args[] = {&x->ctl, &x->conf, &x->gh};
    kp.func = (void *)k_phase3;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(32);
    kp.kernelParams = p3_args;
    if (cudaGraphAddKernelNode(&x->gnode_p3, body, &x->gnode_map, 1, &kp) != cudaSuccess) return TREES_ERR_CUDA;
    if (cudaGraphInstantiate(&x->gexec, x->graph, 0) != cudaSuccess) return TREES_ERR_CUDA;
    return TREES_OK;
}

// Refreshes the Conf argument of the graph's kernels (the job changes per run).
static int update_graph_args(trees_ctx *x) {
    static int from_ctl = 1;
    static uint32_t zero = 0;
    void *ep_args[] = {&x->ctl, &x->conf, &x->blk, &from_ctl, &zero, &zero, &zero, &zero, &zero};
    cudaKernelNodeParams kp;
    std::memset(&kp, 0, sizeof(kp));
    kp.func = const_cast<void *>(x->kern.epoch);
    kp.gridDim = dim3(x->grid);
    kp.blockDim = dim3(x->bs);
    kp.kernelParams = ep_args;
    if (cudaGraphExecKernelNodeSetParams(x->gexec, x->gnode_epoch, &kp) != cudaSuccess) return TREES_ERR_CUDA;
    void *part_args[] = {&x->ctl, &x->conf, &from_ctl, &zero};
    kp.func = const_cast<void *>(x->kern.partition);
    kp.kernelParams = part_args;
    if (cudaGraphExecKernelNodeSetParams(x->gexec, x->gnode_part, &kp) != cudaSuccess) return TREES_ERR_CUDA;
    void *map_args[] = {&x->ctl, &x->conf, &from_ctl, &zero, &zero, &zero};
    kp.func = const_cast<void *>(x->kern.map);
    kp.kernelParams = map_args;
    if (cudaGraphExecKernelNodeSetParams(x->gexec, x->gnode_map, &kp) != cudaSuccess) return TREES_ERR_CUDA;
    void *p3_args[] = {&x->ctl, &x->conf, &x->gh};
    kp.func = (void *)k_phase3;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(32);
    kp.kernelParams = p3_args;
    if (cudaGraphExecKernelNodeSetParams(x->gexec, x->gnode_p3, &kp) != cudaSuccess) return TREES_ERR_CUDA;
    return TREES_OK;
}

// The paper's host loop (Sec. 5.2.2-5.2.4), one launch and one read-back per epoch.
static int run_hostloop(trees_ctx *x, cudaStream_t st) {
    struct R {
        uint32_t cen, lo, hi;
    };
    std::vector<R> stk;
    x->host_trace.clear();
    uint32_t cen = 0, lo = 0, hi = 1, base = 1, e = 0, next = 1, peak = 1;
    unsigned long long forks = 0;
    int status = TREES_OK;
    Ctl *h = x->pinned_ctl;
    for (;;) {
        const uint32_t ep = e % 3u;
        const uint32_t per = (uint32_t)x->bs * (uint32_t)x->cfg.tasks_per_thread;
        const uint32_t nb = (hi - lo + per - 1) / per;
        void *args[] = {&x->ctl, &x->conf, &x->blk, nullptr, &cen, &lo, &hi, &base, &e};
        int from_ctl = 0;
        args[3] = &from_ctl;
        if (cudaLaunchKernel(x->kern.epoch, dim3(nb), dim3(x->bs), args, 0, st) != cudaSuccess) return TREES_ERR_CUDA;
        if (cudaMemcpyAsync(h, x->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st) != cudaSuccess) return TREES_ERR_CUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) return TREES_ERR_CUDA;
        if (h->err) {
            status = h->err;
            break;
        }
        const unsigned long long mt = h->mt_ctr[ep], me = h->me_ctr[ep];
        if (mt | me) {  // mapScheduled: run the map kernel before the next epoch
            if ((uint32_t)(mt & CTR_LOW_MASK) > (uint32_t)(mt >> 40)) {
                void *pargs[] = {&x->ctl, &x->conf, &from_ctl, &e};
                if (cudaLaunchKernel(x->kern.partition, dim3(x->grid), dim3(x->bs), pargs, 0, st) != cudaSuccess)
                    return TREES_ERR_CUDA;
            }
            void *margs[] = {&x->ctl, &x->conf, &from_ctl, &cen, &base, &e};
            if (cudaLaunchKernel(x->kern.map, dim3(x->grid), dim3(x->bs), margs, 0, st) != cudaSuccess)
                return TREES_ERR_CUDA;
            if (cudaMemcpyAsync(h, x->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st) != cudaSuccess)
                return TREES_ERR_CUDA;
            if (cudaStreamSynchronize(st) != cudaSuccess) return TREES_ERR_CUDA;
            if (h->err) {
                status = h->err;
                break;
            }
        }
        const uint32_t f = (uint32_t)(h->ew[ep] >> 32), jf = h->join[ep];
        if (jf) stk.push_back(R{cen, lo, hi});
        if (f) {
            stk.push_back(R{cen + 1u, base, base + f});
            next = base + f;
        } else if (!jf) {
            next = lo;
        }
        forks += f;
        peak = std::max(peak, base + f);
        trees_epoch_t r;
        std::memset(&r, 0, sizeof(r));
        r.cen = cen;
        r.lo = lo;
        r.hi = hi;
        r.forks = f;
        r.joined = jf;
        r.maps = (uint32_t)(mt >> 40) + (uint32_t)(me >> 40);
        if (x->cfg.trace && e < x->cfg.trace_cap) x->host_trace.push_back(r);
        ++e;
        if (stk.size() > STK_CAP) {
            status = TREES_ERR_STACK;
            break;
        }
        if (stk.empty()) break;
        if (e >= x->cfg.max_epochs) {
            status = TREES_ERR_EPOCH_LIMIT;
            break;
        }
        const R r2 = stk.back();
        stk.pop_back();
        cen = r2.cen;
        lo = r2.lo;
        hi = r2.hi;
        base = next;
    }
    // record the run's scheduler-side statistics where trees_stats reads them
    Ctl upd;
    if (cudaMemcpy(&upd, x->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost) != cudaSuccess) return TREES_ERR_CUDA;
    upd.epochs = e;
    upd.peak = peak;
    upd.final_next = next;
    upd.forks = forks;
    if (status != TREES_OK && upd.err == 0) {
        upd.err = status;
        upd.err_epoch = e;
    }
    if (cudaMemcpy(x->ctl, &upd, sizeof(Ctl), cudaMemcpyHostToDevice) != cudaSuccess) return TREES_ERR_CUDA;
    return status;
}

int trees_run(trees_ctx *x, const trees_job_t *job, void *stream) {
    if (!x || !job) return TREES_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    RunParams &rp = x->conf.rp;
    std::memset(&rp, 0, sizeof(rp));
    x->conf.smp = nullptr;
    rp.program = job->program;
    rp.n = job->n;
    rp.cutoff = job->cutoff;
    rp.leaf = job->leaf ? job->leaf : LEAF_MAX;
    uint32_t type = 0, a0 = 0, a1 = 0;
    switch (job->program) {
    case TREES_PROG_FIB:
        if (job->n > 93 || job->cutoff > 30) return TREES_ERR_INVALID_ARG;
        type = TREES_TASK_FIB;
        a0 = job->n;
        break;
    case TREES_PROG_NQUEENS:
        if (job->n < 1 || job->n > 16) return TREES_ERR_INVALID_ARG;
        type = TREES_TASK_NQ_ROW;
        break;
    case TREES_PROG_MERGESORT:
        if (rp.leaf > (uint32_t)LEAF_MAX || (job->n && !job->keys)) return TREES_ERR_INVALID_ARG;
        rp.keys = job->keys;
        rp.scratch = job->scratch;
        if (!rp.scratch && job->n) {
            if (x->own_scratch_n < job->n) {
                if (x->own_scratch) cudaFree(x->own_scratch);
                x->own_scratch = nullptr;
                x->own_scratch_n = 0;
                if (cudaMalloc(&x->own_scratch, (size_t)job->n * 4) != cudaSuccess) return TREES_ERR_CUDA;
                x->own_scratch_n = job->n;
            }
            rp.scratch = x->own_scratch;
        }
        if (job->n >= (1u << 16)) {  // splitter samples for the partition searches of long runs
            const size_t ns = ((size_t)job->n >> SMP_SHIFT) + 1;
            if (x->own_smp_n < ns) {
                if (x->own_smp) cudaFree(x->own_smp);
                x->own_smp = nullptr;
                x->own_smp_n = 0;
                if (cudaMalloc(&x->own_smp, ns * 4) != cudaSuccess) return TREES_ERR_CUDA;
                x->own_smp_n = ns;
            }
            x->conf.smp = x->own_smp;
        }
        type = TREES_TASK_MS_SPLIT;
        a0 = 0;
        a1 = job->n;
        break;
    case TREES_PROG_BFS:
        if (!job->row_ptr || !job->level || job->nv < 1 || (int32_t)job->n < 0 || (int32_t)job->n >= job->nv)
            return TREES_ERR_INVALID_ARG;
        rp.row_ptr = job->row_ptr;
        rp.col = job->col;
        rp.level = job->level;
        rp.nv = job->nv;
        {  // the visited bits: the context's per-vertex buffer, which BFS does not use otherwise
            const size_t words = ((size_t)job->nv + 63) / 64;
            if (x->own_used_n < words) {
                if (x->own_used) cudaFree(x->own_used);
                x->own_used = nullptr;
                x->own_used_n = 0;
                if (cudaMalloc(&x->own_used, words * 8) != cudaSuccess) return TREES_ERR_CUDA;
                x->own_used_n = words;
            }
            rp.visited = reinterpret_cast<uint32_t *>(x->own_used);
        }
        type = TREES_TASK_BFS_VISIT;
        a0 = job->n;
        break;
    case TREES_PROG_SSSP:
        if (!job->row_ptr || !job->col || !job->weight || !job->dist || !job->sched || job->nv < 1 ||
            (int32_t)job->n < 0 || (int32_t)job->n >= job->nv)
            return TREES_ERR_INVALID_ARG;
        rp.row_ptr = job->row_ptr;
        rp.col = job->col;
        rp.weight = job->weight;
        rp.dist = reinterpret_cast<unsigned long long *>(job->dist);
        rp.sched = job->sched;
        rp.nv = job->nv;
        if (x->own_used_n < (size_t)job->nv) {  // the relax records, one word per vertex, owned by the context
            if (x->own_used) cudaFree(x->own_used);
            x->own_used = nullptr;
            x->own_used_n = 0;
            if (cudaMalloc(&x->own_used, (size_t)job->nv * 8) != cudaSuccess) return TREES_ERR_CUDA;
            x->own_used_n = (size_t)job->nv;
        }
        rp.used = x->own_used;
        type = TREES_TASK_SSSP_RELAX;
        a0 = job->n;
        break;
    case TREES_PROG_FFT: {
        const uint32_t n = job->n, leaf = job->leaf ? job->leaf : FFT_LEAF_MAX;
        const uintptr_t in = (uintptr_t)job->fft_in, out = (uintptr_t)job->fft_out, bytes = (uintptr_t)n * 8u;
        if (n < 1u || (n & (n - 1u)) || n > FFT_MAX_POINTS || leaf > FFT_LEAF_MAX || (leaf & (leaf - 1u)) || !in ||
            !out || (in & 7u) || (out & 7u) || (in < out + bytes && out < in + bytes))
            return TREES_ERR_INVALID_ARG;
        rp.leaf = leaf;
        rp.fx = reinterpret_cast<const float2 *>(job->fft_in);
        rp.fX = reinterpret_cast<float2 *>(job->fft_out);
        rp.lgn = (uint32_t)__builtin_ctz(n);
        type = TREES_TASK_FFT;
        a0 = 0;
        a1 = 0;
        break;
    }
    case TREES_PROG_USER:  // its own kernel, launched through its function: persistent scheduler only
        if (!job->user_program || job->user_type < 1u || job->user_type > (uint32_t)TREES_NUM_TASK_TYPES ||
            x->cfg.scheduler != TREES_SCHED_PERSISTENT)
            return TREES_ERR_INVALID_ARG;
        for (int i = 0; i < TREES_USER_PARAMS; ++i) {
            rp.up[i] = job->user_ptr[i];
            rp.uv[i] = job->user_val[i];
        }
        type = job->user_type;
        a0 = job->user_a0;
        a1 = job->user_a1;
        break;
    case TREES_PROG_POSTORDER:
    case TREES_PROG_PREORDER:
        if (job->n && (!job->left || !job->right || !job->visit_epoch)) return TREES_ERR_INVALID_ARG;
        rp.left = job->left;
        rp.right = job->right;
        rp.visit_epoch = job->visit_epoch;
        type = job->program == TREES_PROG_POSTORDER ? TREES_TASK_PO : TREES_TASK_PRE;
        a0 = job->n ? 0u : 0xFFFFFFFFu;
        break;
    default:
        return TREES_ERR_INVALID_ARG;
    }
    x->last_stream = st;
    x->res0_valid = false;
    x->last_sched = x->cfg.scheduler;
    // the library's persistent kernels copy slot 0's result beside the status word at their end; a
    // user program's kernel (built from the same headers in its own library) is not relied on
    x->res0_in_ctl = x->cfg.scheduler == TREES_SCHED_PERSISTENT && job->program != TREES_PROG_USER;
    if (x->cfg.trace && cudaMemsetAsync(x->conf.trace_valid, 0, (size_t)x->cfg.trace_cap * 4, st) != cudaSuccess)
        return TREES_ERR_CUDA;
    k_setup<<<SETUP_BLOCKS, 256, 0, st>>>(x->ctl, x->conf, type, a0, a1, x->blk);
    if (job->program == TREES_PROG_BFS) {
        const int nb = std::min<int64_t>((job->nv + 255) / 256, 65536);
        k_bfs_init<<<nb, 256, 0, st>>>(job->level, rp.visited, job->nv, (int32_t)job->n);
    }
    if (job->program == TREES_PROG_SSSP) {
        const int nb = std::min<int64_t>((job->nv + 255) / 256, 65536);
        k_sssp_init<<<nb, 256, 0, st>>>(rp.dist, job->sched, rp.used, job->nv, (int32_t)job->n);
    }
    if (job->program == TREES_PROG_POSTORDER || job->program == TREES_PROG_PREORDER) {
        if (job->n && cudaMemsetAsync(job->visit_epoch, 0xFF, (size_t)job->n * 4, st) != cudaSuccess)
            return TREES_ERR_CUDA;
    }
    if (cudaGetLastError() != cudaSuccess) return TREES_ERR_CUDA;
    switch (x->cfg.scheduler) {
    case TREES_SCHED_PERSISTENT: {
        void *args[] = {&x->ctl, &x->conf, &x->blk};
        if (job->program == TREES_PROG_USER) {
            const trees_program_fn f = job->user_program;
            int32_t occ = 0;
            if (f(TREES_USER_OP_OCCUPANCY, x->bs, x->cfg.tasks_per_thread, nullptr, 0, stream, &occ) != 0 || occ < 1)
                return TREES_ERR_CUDA;
            const int per_sm = x->cfg.blocks_per_sm > 0 ? std::min(x->cfg.blocks_per_sm, (int)occ) : (int)occ;
            const int grid = x->cfg.grid_blocks > 0 ? std::min(x->cfg.grid_blocks, x->sms * (int)occ) : x->sms * per_sm;
            x->last_grid = grid;
            if (f(TREES_USER_OP_LAUNCH, x->bs, x->cfg.tasks_per_thread, args, grid, stream, nullptr) != 0) {
                cudaGetLastError();
                return TREES_ERR_CUDA;
            }
            return TREES_OK;
        }
        const void *kern = persistent_kernel(job->program, x->bs, x->cfg.tasks_per_thread);
        const size_t smem = persistent_smem_bytes(program_mask(job->program), x->bs, x->cfg.tasks_per_thread);
        const int grid = kernel_grid(x, kern, smem);
        if (!kern || grid < 1) return TREES_ERR_CUDA;
        x->last_grid = grid;
        if (cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(x->bs), args, smem, st) != cudaSuccess) {
            cudaGetLastError();
            return TREES_ERR_CUDA;
        }
        return TREES_OK;
    }
    case TREES_SCHED_GRAPH: {
        int rc = build_graph(x);
        if (rc) return rc;
        rc = update_graph_args(x);
        if (rc) return rc;
        if (cudaGraphLaunch(x->gexec, st) != cudaSuccess) return TREES_ERR_CUDA;
        return TREES_OK;
    }
    case TREES_SCHED_HOSTLOOP: {
        const int rc = run_hostloop(x, st);
        x->host_status = rc;
        return (rc == TREES_ERR_CUDA || rc == TREES_ERR_INVALID_ARG) ? rc : TREES_OK;
    }
    }
    return TREES_ERR_INVALID_ARG;
}

// The run's status and its root result (slot 0, where fib and N-Queens
// leave theirs) follow the run on its stream into pinned host memory, so the
// host waits once instead of once per synchronous copy; trees_result(x, 0)
// then returns the copied value until the next run.  After a persistent run
// the kernel has put the result beside the status word, and one 16-byte copy
// brings both (fib(34) end to end: 0.4168 -> 0.4157 ms per step).
static_assert(offsetof(Ctl, res0) == offsetof(Ctl, err) + 8 && offsetof(trees_ctx::SyncPin, res0) == 8,
              "status word and slot 0's result copy as one block");
int trees_sync(trees_ctx *x) {
    if (!x) return TREES_ERR_INVALID_ARG;
    if (x->res0_in_ctl) {
        if (cudaMemcpyAsync(x->pin_sync, &x->ctl->err, 16, cudaMemcpyDeviceToHost, x->last_stream) != cudaSuccess)
            return TREES_ERR_CUDA;
    } else if (cudaMemcpyAsync(&x->pin_sync->err, &x->ctl->err, sizeof(int), cudaMemcpyDeviceToHost,
                               x->last_stream) != cudaSuccess ||
               cudaMemcpyAsync(&x->pin_sync->res0, x->conf.result, 8, cudaMemcpyDeviceToHost, x->last_stream) !=
                   cudaSuccess) {
        return TREES_ERR_CUDA;
    }
    if (cudaStreamSynchronize(x->last_stream) != cudaSuccess) return TREES_ERR_CUDA;
    x->res0_valid = true;
    return x->pin_sync->err;
}

int trees_result(trees_ctx *x, uint32_t slot, uint64_t *out) {
    if (!x || !out || slot >= x->cap) return TREES_ERR_INVALID_ARG;
    if (slot == 0u && x->res0_valid) {  // copied by trees_sync after the last run
        *out = x->pin_sync->res0;
        return TREES_OK;
    }
    unsigned long long v = 0;
    if (cudaMemcpy(&v, x->conf.result + slot, 8, cudaMemcpyDeviceToHost) != cudaSuccess) return TREES_ERR_CUDA;
    *out = v;
    return TREES_OK;
}

int trees_stats(trees_ctx *x, trees_stats_t *out) {
    if (!x || !out) return TREES_ERR_INVALID_ARG;
    Ctl h;
    if (cudaMemcpy(&h, x->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost) != cudaSuccess) return TREES_ERR_CUDA;
    std::vector<unsigned long long> blk((size_t)NBLK_STATS * 4);
    if (cudaMemcpy(blk.data(), x->blk, blk.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess) return TREES_ERR_CUDA;
    unsigned long long tasks = 0, joins = 0, maps = 0;
    for (int b = 0; b < NBLK_STATS; ++b) {
        tasks += blk[4 * b + 0];
        joins += blk[4 * b + 1];
        maps += blk[4 * b + 2];
    }
    out->epochs = h.epochs;
    out->tasks = tasks;
    out->forks = h.forks;
    out->joins = joins;
    out->maps = maps;
    out->peak_slots = h.peak;
    out->final_slots = h.final_next;
    out->ns = h.t_end > h.t_start ? h.t_end - h.t_start : 0;
    out->status = h.err;
    out->error_epoch = (int32_t)h.err_epoch;
    out->grid_blocks = x->last_sched == TREES_SCHED_PERSISTENT && x->last_grid ? x->last_grid : x->grid;
    out->block_size = x->bs;
    return TREES_OK;
}

int trees_trace(trees_ctx *x, trees_epoch_t *out, size_t cap, size_t *n) {
    if (!x || (!out && cap) || !n) return TREES_ERR_INVALID_ARG;
    Ctl h;
    if (cudaMemcpy(&h, x->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost) != cudaSuccess) return TREES_ERR_CUDA;
    size_t m = std::min<size_t>({cap, (size_t)h.epochs, (size_t)x->cfg.trace_cap});
    if (!x->cfg.trace) m = 0;
    std::vector<uint32_t> valid(m);
    if (m) {
        if (x->last_sched == TREES_SCHED_HOSTLOOP) {
            m = std::min(m, x->host_trace.size());
            std::memcpy(out, x->host_trace.data(), m * sizeof(trees_epoch_t));
        } else if (cudaMemcpy(out, x->conf.trace, m * sizeof(trees_epoch_t), cudaMemcpyDeviceToHost) != cudaSuccess) {
            return TREES_ERR_CUDA;
        }
        if (cudaMemcpy(valid.data(), x->conf.trace_valid, m * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
            return TREES_ERR_CUDA;
        for (size_t i = 0; i < m; ++i) out[i].valid = valid[i];
    }
    *n = m;
    return TREES_OK;
}

int trees_fib(trees_ctx *x, uint32_t n, uint32_t cutoff, void *stream) {
    trees_job_t j;
    std::memset(&j, 0, sizeof(j));
    j.program = TREES_PROG_FIB;
    j.n = n;
    j.cutoff = cutoff;
    return trees_run(x, &j, stream);
}

int trees_nqueens(trees_ctx *x, uint32_t n, void *stream) {
    trees_job_t j;
    std::memset(&j, 0, sizeof(j));
    j.program = TREES_PROG_NQUEENS;
    j.n = n;
    return trees_run(x, &j, stream);
}

int trees_mergesort_u32(trees_ctx *x, uint32_t *keys, uint32_t *scratch, uint32_t n, void *stream) {
    trees_job_t j;
    std::memset(&j, 0, sizeof(j));
    j.program = TREES_PROG_MERGESORT;
    j.n = n;
    j.keys = keys;
    j.scratch = scratch;
    return trees_run(x, &j, stream);
}

int trees_bfs(trees_ctx *x, const int32_t *row_ptr, const int32_t *col, int32_t nv, int32_t src, int32_t *level,
              void *stream) {
    trees_job_t j;
    std::memset(&j, 0, sizeof(j));
    j.program = TREES_PROG_BFS;
    j.n = (uint32_t)src;
    j.row_ptr = row_ptr;
    j.col = col;
    j.nv = nv;
    j.level = level;
    return trees_run(x, &j, stream);
}

int trees_sssp(trees_ctx *x, const int32_t *row_ptr, const int32_t *col, const uint32_t *weight, int32_t nv,
               int32_t src, uint64_t *dist, uint32_t *sched, void *stream) {
    trees_job_t j;
    std::memset(&j, 0, sizeof(j));
    j.program = TREES_PROG_SSSP;
    j.n = (uint32_t)src;
    j.row_ptr = row_ptr;
    j.col = col;
    j.weight = weight;
    j.nv = nv;
    j.dist = dist;
    j.sched = sched;
    return trees_run(x, &j, stream);
}

int trees_fft(trees_ctx *x, const float *in, float *out, uint32_t n, uint32_t leaf, uint32_t cutoff, void *stream) {
    trees_job_t j;
    std::memset(&j, 0, sizeof(j));
    j.program = TREES_PROG_FFT;
    j.n = n;
    j.leaf = leaf;
    j.cutoff = cutoff;
    j.fft_in = in;
    j.fft_out = out;
    return trees_run(x, &j, stream);
}

int trees_barrier_floor(trees_ctx *x, uint32_t iters, void *stream, double *us) {
    if (!x || !us || iters == 0) return TREES_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return TREES_ERR_CUDA;
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return TREES_ERR_CUDA;
    }
    int rc = TREES_OK;
    unsigned long long to = x->cfg.timeout_ns;
    void *args[] = {&x->ctl, &iters, &to};
    if (cudaMemsetAsync(x->ctl, 0, sizeof(Ctl), st) != cudaSuccess ||
        cudaEventRecord(a, st) != cudaSuccess ||
        cudaLaunchCooperativeKernel(x->kern.floor, dim3(x->last_grid ? x->last_grid : x->grid), dim3(x->bs), args, 0,
                                    st) != cudaSuccess ||
        cudaEventRecord(b, st) != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess) {
        cudaGetLastError();
        rc = TREES_ERR_CUDA;
    }
    if (!rc) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        *us = 1000.0 * ms / iters;
        int err = 0;
        cudaMemcpy(&err, &x->ctl->err, sizeof(int), cudaMemcpyDeviceToHost);
        if (err) rc = err;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return rc;
}

}  // extern "C"

// ------------------------------------------------------------------ allocation-free fib entry point
//
// Some callers cannot allocate device memory at call time: code running
// under a CUDA stream capture that must not allocate, real-time or embedded
// hosts whose memory budget is fixed at start-up, and plugins whose host
// application owns the allocator.  trees_fib_noalloc serves them: it runs the
// persistent epoch kernel with its task vector, control block and statistics
// carved out of one file-scope device array below, so it never calls
// cudaMalloc, cudaFree or any allocating routine.  The array (NOALLOC_BYTES)
// is part of the library image: every GPU that loads libtrees keeps it until
// the process exits.  All calls share it and it keeps the previous call's
// contents; the control block and statistics are cleared at the start of
// each call.  Two calls whose work overlaps on the GPU race on the array, so
// a caller must order them (one stream, or a stream/event dependency).

namespace {

constexpr size_t NOALLOC_CAP = 1u << 20;        // task-vector slots: fib(n) needs 2F(n+1)-1
constexpr size_t NOALLOC_BYTES = 26u << 20;     // 26 MiB: TV columns (24 MiB) + control block, lists, stats

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

struct NoallocDevice {
    std::mutex mu;         // serialises the set-up of host threads making a first call at once
    bool ready = false;    // written under mu; read under mu
    char *base = nullptr;  // device address of g_noalloc_scratch on this device
    int grid = 0, sms = 0;
};
NoallocDevice g_noalloc_dev[64];

// Once per device, with that device current: find the device address of the
// static array (host code only sees a host-side stand-in for the symbol) and
// the cooperative grid size.  Threads that race on a device's first call
// wait on its mutex; a set-up that failed is tried again by the next call.
int noalloc_setup(int dev, NoallocDevice *d) {
    std::lock_guard<std::mutex> lock(d->mu);
    if (d->ready) return TREES_OK;
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
        cudaGetLastError();
        return TREES_ERR_CUDA;
    }
    int sms = 0, occ = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return TREES_ERR_CUDA;
    const size_t smem = persistent_smem_bytes(PM_FIB, 1024, 2);
    if (smem && cudaFuncSetAttribute(persistent_kernel_fib(1024, 2), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return TREES_ERR_CUDA;
    }
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, persistent_kernel_fib(1024, 2), 1024, smem) !=
            cudaSuccess || occ < 1)
        return TREES_ERR_CUDA;
    if (make_layout(NOALLOC_CAP, 1, 1, STK_CAP).total > NOALLOC_BYTES) return TREES_ERR_CUDA;
    d->base = static_cast<char *>(p);
    d->sms = sms;
    d->grid = sms * occ;
    d->ready = true;
    return TREES_OK;
}

}  // namespace

extern "C" int trees_fib_noalloc(uint32_t n, uint32_t cutoff, uint64_t *dev_result, int32_t *dev_status,
                                 void *stream) {
    if (!dev_result || !dev_status || n > 93 || cutoff > 30) return TREES_ERR_INVALID_ARG;
    // slots the task tree needs at its peak: every node of the tree, where a
    // node of size k is a leaf when k < 2 or k <= cutoff (saturating count)
    uint64_t nk2 = 1, nk1 = 1, need = 1;
    for (uint32_t k = 0; k <= n; ++k) {
        need = (k < 2 || k <= cutoff) ? 1 : std::min<uint64_t>(1 + nk1 + nk2, NOALLOC_CAP + 1);
        nk2 = nk1;
        nk1 = need;
    }
    if (need > NOALLOC_CAP) return TREES_ERR_CAPACITY;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return TREES_ERR_CUDA;
    NoallocDevice *d = &g_noalloc_dev[dev];
    const int rc = noalloc_setup(dev, d);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const Layout L = make_layout(NOALLOC_CAP, 1, 1, STK_CAP);
    char *m0 = d->base;
    Ctl *ctl = reinterpret_cast<Ctl *>(m0 + L.off_dev);
    Conf c;
    std::memset(&c, 0, sizeof(c));
    c.code = reinterpret_cast<uint32_t *>(m0 + L.off_code);
    c.a0 = reinterpret_cast<uint32_t *>(m0 + L.off_a0);
    c.a1 = reinterpret_cast<uint32_t *>(m0 + L.off_a1);
    c.link = reinterpret_cast<uint32_t *>(m0 + L.off_link);
    c.result = reinterpret_cast<unsigned long long *>(m0 + L.off_result);
    c.cap = (uint32_t)NOALLOC_CAP;
    uint32_t **mt[NMT] = {&c.mt_kind, &c.mt_a, &c.mt_b, &c.mt_c, &c.mt_job, &c.mt_tilebase, &c.mt_split};
    for (int i = 0; i < NMT; ++i) *mt[i] = reinterpret_cast<uint32_t *>(m0 + L.off_mt[i]);
    uint32_t **me[NME] = {&c.me_v, &c.me_base, &c.me_job, &c.me_tfd, &c.me_src};
    for (int i = 0; i < NME; ++i) *me[i] = reinterpret_cast<uint32_t *>(m0 + L.off_me[i]);
    c.mcap = 1;
    c.trace = reinterpret_cast<trees_epoch_t *>(m0 + L.off_trace);
    c.trace_valid = reinterpret_cast<uint32_t *>(m0 + L.off_tvalid);
    c.trace_cap = 1;
    c.trace_on = 0;
    c.max_epochs = 1u << 20;
    c.stall_epoch = -1;
    c.timeout_ns = 2000000000ull;
    c.gstack = reinterpret_cast<Range *>(m0 + L.off_gstack);
    c.gstack_cap = STK_CAP;
    c.rp.program = TREES_PROG_FIB;
    c.rp.n = n;
    c.rp.cutoff = cutoff;
    c.rp.leaf = LEAF_MAX;
    unsigned long long *blk = reinterpret_cast<unsigned long long *>(m0 + L.off_blk);
    k_setup<<<SETUP_BLOCKS, 256, 0, st>>>(ctl, c, TREES_TASK_FIB, n, 0u, blk);
    if (cudaGetLastError() != cudaSuccess) return TREES_ERR_CUDA;
    void *args[] = {&ctl, &c, &blk};
    if (cudaLaunchCooperativeKernel(persistent_kernel_fib(1024, 2), dim3(d->grid), dim3(1024), args,
                                    persistent_smem_bytes(PM_FIB, 1024, 2), st) !=
        cudaSuccess) {
        cudaGetLastError();
        return TREES_ERR_CUDA;
    }
    if (cudaMemcpyAsync(dev_result, c.result, sizeof(uint64_t), cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(dev_status, &ctl->err, sizeof(int32_t), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return TREES_ERR_CUDA;
    return TREES_OK;
}

// ------------------------------------------------------------------ batches and serving (host)

namespace {

// Peak task-vector need of one job (see trees_job_slots).
uint64_t job_slots(const trees_job_t *j, int32_t *exact) {
    int32_t ex = 1;
    uint64_t need = 1;
    switch (j->program) {
    case TREES_PROG_FIB: {  // every node of the fib tree is resident at the peak
        uint64_t nk2 = 1, nk1 = 1;
        for (uint32_t k = 0; k <= j->n; ++k) {
            need = (k < 2 || k <= j->cutoff) ? 1 : std::min<uint64_t>(1 + nk1 + nk2, 1ull << 40);
            nk2 = nk1;
            nk1 = need;
        }
        break;
    }
    case TREES_PROG_MERGESORT: {  // every split node of the tree
        const uint64_t leaf = j->leaf ? j->leaf : LEAF_MAX;
        std::map<uint64_t, uint64_t> memo;
        struct F {
            static uint64_t go(uint64_t m, uint64_t leaf, std::map<uint64_t, uint64_t> &memo) {
                if (m <= leaf) return 1;
                auto it = memo.find(m);
                if (it != memo.end()) return it->second;
                const uint64_t h = m / 2, r = 1 + go(h, leaf, memo) + go(m - h, leaf, memo);
                memo[m] = r;
                return r;
            }
        };
        need = F::go(j->n, leaf, memo);
        break;
    }
    case TREES_PROG_NQUEENS: {  // estimate 4 * 3^(n-1); a job that outgrows it ends with CAPACITY
        ex = 0;
        need = 4;
        for (uint32_t k = 1; k < j->n && need < (1ull << 40); ++k) need *= 3;
        break;
    }
    case TREES_PROG_POSTORDER:
    case TREES_PROG_PREORDER:
        need = 2ull * j->n + 1;  // every node and every nil child
        break;
    case TREES_PROG_BFS:
        need = (uint64_t)std::max(j->nv, 1);
        break;
    case TREES_PROG_SSSP:  // at least one relax task per reachable vertex; more when distances drop again
        need = (uint64_t)std::max(j->nv, 1);
        ex = 0;
        break;
    case TREES_PROG_FFT: {  // the whole task tree: 2^(D+1) - 1 FFT tasks, D = log2(n / leaf)
        const uint64_t leaf = j->leaf ? j->leaf : FFT_LEAF_MAX;
        uint64_t D = 0;
        while (((uint64_t)j->n >> D) > leaf) ++D;
        need = (2ull << D) - 1ull;
        break;
    }
    default:
        need = 0;
        ex = 0;
    }
    if (exact) *exact = ex;
    return need;
}

// Validates a job for batched execution and fills its table record.
int make_job_record(const trees_job_t *j, uint32_t seg_base, uint32_t seg_cap, uint64_t id, Job *r) {
    std::memset(r, 0, sizeof(Job));
    RunParams &rp = r->rp;
    rp.program = j->program;
    rp.n = j->n;
    rp.cutoff = j->cutoff;
    rp.leaf = j->leaf ? j->leaf : LEAF_MAX;
    switch (j->program) {
    case TREES_PROG_FIB:
        if (j->n > 93 || j->cutoff > 30) return TREES_ERR_INVALID_ARG;
        r->type0 = TREES_TASK_FIB;
        r->a00 = j->n;
        break;
    case TREES_PROG_NQUEENS:
        if (j->n < 1 || j->n > 16) return TREES_ERR_INVALID_ARG;
        r->type0 = TREES_TASK_NQ_ROW;
        break;
    case TREES_PROG_MERGESORT:
        if (rp.leaf > (uint32_t)LEAF_MAX || (j->n && (!j->keys || !j->scratch))) return TREES_ERR_INVALID_ARG;
        rp.keys = j->keys;
        rp.scratch = j->scratch;
        r->type0 = TREES_TASK_MS_SPLIT;
        r->a10 = j->n;
        break;
    case TREES_PROG_POSTORDER:
    case TREES_PROG_PREORDER:
        if (j->n && (!j->left || !j->right || !j->visit_epoch)) return TREES_ERR_INVALID_ARG;
        rp.left = j->left;
        rp.right = j->right;
        rp.visit_epoch = j->visit_epoch;
        r->type0 = j->program == TREES_PROG_POSTORDER ? TREES_TASK_PO : TREES_TASK_PRE;
        r->a00 = j->n ? 0u : 0xFFFFFFFFu;
        break;
    default:
        return TREES_ERR_INVALID_ARG;  // BFS runs through trees_run only
    }
    r->seg_base = seg_base;
    r->seg_cap = seg_cap;
    r->state = JOB_NEW;
    r->id = id;
    return TREES_OK;
}

template <int BS>
const void *batch_kernel() {
    return (const void *)k_batch<BS>;
}

const void *batch_kernel_for(int bs) {
    switch (bs) {
    case 128: return batch_kernel<128>();
    case 256: return batch_kernel<256>();
    case 512: return batch_kernel<512>();
    default: return batch_kernel<1024>();
    }
}

int batch_grid(trees_ctx *x, const void *kern) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, x->bs, 0) != cudaSuccess || occ < 1) return 0;
    const int per_sm = x->cfg.blocks_per_sm > 0 ? std::min(x->cfg.blocks_per_sm, occ) : occ;
    int g = x->sms * per_sm;
    if (x->cfg.grid_blocks > 0) g = std::min(x->cfg.grid_blocks, x->sms * occ);
    return g;
}

int ensure_batch_buffers(trees_ctx *x, int32_t n) {
    if (x->batch_cap >= n) return TREES_OK;
    if (x->d_jobs) cudaFree(x->d_jobs);
    if (x->d_joff) cudaFree(x->d_joff);
    if (x->d_done) cudaFree(x->d_done);
    if (x->d_bc) cudaFree(x->d_bc);
    if (x->h_jobs) cudaFreeHost(x->h_jobs);
    x->d_jobs = nullptr;
    x->d_joff = nullptr;
    x->d_done = nullptr;
    x->d_bc = nullptr;
    x->h_jobs = nullptr;
    x->batch_cap = 0;
    if (cudaMalloc(&x->d_jobs, sizeof(Job) * (size_t)n) != cudaSuccess ||
        cudaMalloc(&x->d_joff, sizeof(uint32_t) * ((size_t)n + 1)) != cudaSuccess ||
        cudaMalloc(&x->d_done, sizeof(BatchDone) * (size_t)n) != cudaSuccess ||
        cudaMalloc(&x->d_bc, sizeof(BatchCtl)) != cudaSuccess ||
        cudaMallocHost(&x->h_jobs, sizeof(Job) * (size_t)n) != cudaSuccess) {
        cudaGetLastError();
        return TREES_ERR_CUDA;
    }
    x->batch_cap = n;
    return TREES_OK;
}

int launch_batch(trees_ctx *x, BatchCtl *d_bc, Job *d_jobs, uint32_t *d_joff, BatchDone *d_done, uint32_t max_steps,
                 cudaStream_t st) {
    const void *kern = batch_kernel_for(x->bs);
    const int grid = batch_grid(x, kern);
    if (grid < 1) return TREES_ERR_CUDA;
    if (cudaMemsetAsync(x->ctl, 0, sizeof(Ctl), st) != cudaSuccess) return TREES_ERR_CUDA;
    void *args[] = {&x->ctl, &x->conf, &d_bc, &d_jobs, &d_joff, &d_done, &max_steps, &x->blk};
    if (cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(x->bs), args, 0, st) != cudaSuccess) {
        cudaGetLastError();
        return TREES_ERR_CUDA;
    }
    return TREES_OK;
}

void fill_result(const BatchDone &d, trees_job_result_t *o) {
    o->id = d.id;
    o->result = d.result;
    o->tasks = d.tasks;
    o->joins = d.joins;
    o->maps = d.maps;
    o->ns = d.ns;
    o->epochs = d.epochs;
    o->peak_slots = d.peak;
    o->status = d.status;
    o->pad = 0;
}

}  // namespace

extern "C" uint64_t trees_job_slots(const trees_job_t *job, int32_t *exact) {
    if (!job) {
        if (exact) *exact = 0;
        return 0;
    }
    return job_slots(job, exact);
}

extern "C" int trees_batch_run(trees_ctx *x, const trees_job_t *jobs, const uint64_t *seg_slots, int32_t njobs,
                               void *stream) {
    if (!x || !jobs || njobs <= 0) return TREES_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = ensure_batch_buffers(x, njobs);
    if (rc) return rc;
    uint64_t base = 0;
    for (int32_t i = 0; i < njobs; ++i) {
        const uint64_t want = seg_slots ? seg_slots[i] : job_slots(&jobs[i], nullptr);
        if (want == 0 || want > 0xFFFFFFFFull) return TREES_ERR_INVALID_ARG;
        if (base + want > x->cap) return TREES_ERR_ADMISSION;
        rc = make_job_record(&jobs[i], (uint32_t)base, (uint32_t)want, (uint64_t)i, &x->h_jobs[i]);
        if (rc) return rc;
        base += want;
    }
    BatchCtl hb;
    std::memset(&hb, 0, sizeof(hb));
    hb.njobs = (unsigned int)njobs;
    hb.max_epochs = x->cfg.max_epochs;
    if (cudaMemcpyAsync(x->d_jobs, x->h_jobs, sizeof(Job) * (size_t)njobs, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(x->d_bc, &hb, sizeof(hb), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return TREES_ERR_CUDA;
    x->last_stream = st;
    x->res0_valid = false;
    x->res0_in_ctl = false;
    x->batch_n = njobs;
    // the host copies above read pageable/pinned host memory; keep hb alive until issued
    if (cudaStreamSynchronize(st) != cudaSuccess) return TREES_ERR_CUDA;
    return launch_batch(x, x->d_bc, x->d_jobs, x->d_joff, x->d_done, 0xFFFFFFFFu, st);
}

extern "C" int trees_batch_results(trees_ctx *x, trees_job_result_t *out, int32_t njobs, uint32_t *steps) {
    if (!x || !out || njobs != x->batch_n) return TREES_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(x->last_stream) != cudaSuccess) return TREES_ERR_CUDA;
    BatchCtl hb;
    int err = 0;
    if (cudaMemcpy(&hb, x->d_bc, sizeof(hb), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&err, &x->ctl->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return TREES_ERR_CUDA;
    std::vector<BatchDone> d(hb.done_count);
    if (hb.done_count && cudaMemcpy(d.data(), x->d_done, sizeof(BatchDone) * hb.done_count,
                                    cudaMemcpyDeviceToHost) != cudaSuccess)
        return TREES_ERR_CUDA;
    for (int32_t i = 0; i < njobs; ++i) {
        std::memset(&out[i], 0, sizeof(out[i]));
        out[i].id = (uint64_t)i;
        out[i].status = err ? err : TREES_ERR_EPOCH_LIMIT;  // overwritten by the job's completion record
    }
    for (const BatchDone &r : d)
        if (r.job < (uint32_t)njobs) fill_result(r, &out[r.job]);
    if (steps) *steps = hb.steps;
    return err;
}

// ------------------------------------------------------------------ server

struct trees_server {
    trees_ctx *ctx = nullptr;
    int32_t max_jobs = 0, steps = 0;
    Job *d_jobs = nullptr, *d_stage = nullptr, *h_stage = nullptr;
    uint32_t *d_joff = nullptr, *d_entries = nullptr, *h_entries = nullptr;
    BatchDone *d_done = nullptr, *h_done = nullptr;
    BatchCtl *d_bc = nullptr, *h_bc = nullptr;
    struct Pending {
        trees_job_t job;
        uint64_t slots, id;
    };
    std::deque<Pending> queue;
    std::vector<int32_t> free_entries;
    std::vector<uint8_t> used;
    std::vector<std::pair<uint32_t, uint32_t>> seg;  // per entry: base, length
    std::map<uint32_t, uint32_t> free_seg;           // base -> length
    std::vector<trees_job_result_t> finished;
    uint32_t hw = 0;
    int32_t running = 0;
    uint64_t next_id = 0, launches = 0;
};

namespace {

bool seg_alloc(trees_server *s, uint32_t len, uint32_t *base) {
    for (auto it = s->free_seg.begin(); it != s->free_seg.end(); ++it) {
        if (it->second >= len) {
            *base = it->first;
            const uint32_t rest = it->second - len, nb = it->first + len;
            s->free_seg.erase(it);
            if (rest) s->free_seg[nb] = rest;
            return true;
        }
    }
    return false;
}

void seg_free(trees_server *s, uint32_t base, uint32_t len) {
    auto it = s->free_seg.emplace(base, len).first;
    auto nx = std::next(it);
    if (nx != s->free_seg.end() && it->first + it->second == nx->first) {
        it->second += nx->second;
        s->free_seg.erase(nx);
    }
    if (it != s->free_seg.begin()) {
        auto pv = std::prev(it);
        if (pv->first + pv->second == it->first) {
            pv->second += it->second;
            s->free_seg.erase(it);
        }
    }
}

}  // namespace

extern "C" int trees_server_create(size_t pool_slots, int32_t max_jobs, int32_t steps_per_launch,
                                   const trees_config_t *cfg, trees_server **out) {
    if (!out || max_jobs <= 0 || steps_per_launch <= 0) return TREES_ERR_INVALID_ARG;
    *out = nullptr;
    trees_server *s = new (std::nothrow) trees_server();
    if (!s) return TREES_ERR_INVALID_ARG;
    int rc = trees_create(pool_slots, cfg, &s->ctx);
    if (rc) {
        delete s;
        return rc;
    }
    s->max_jobs = max_jobs;
    s->steps = steps_per_launch;
    const size_t n = (size_t)max_jobs;
    if (cudaMalloc(&s->d_jobs, sizeof(Job) * n) != cudaSuccess || cudaMalloc(&s->d_stage, sizeof(Job) * n) != cudaSuccess ||
        cudaMalloc(&s->d_joff, sizeof(uint32_t) * (n + 1)) != cudaSuccess ||
        cudaMalloc(&s->d_entries, sizeof(uint32_t) * n) != cudaSuccess ||
        cudaMalloc(&s->d_done, sizeof(BatchDone) * n) != cudaSuccess ||
        cudaMalloc(&s->d_bc, sizeof(BatchCtl)) != cudaSuccess ||
        cudaMallocHost(&s->h_stage, sizeof(Job) * n) != cudaSuccess ||
        cudaMallocHost(&s->h_entries, sizeof(uint32_t) * n) != cudaSuccess ||
        cudaMallocHost(&s->h_done, sizeof(BatchDone) * n) != cudaSuccess ||
        cudaMallocHost(&s->h_bc, sizeof(BatchCtl)) != cudaSuccess ||
        cudaMemset(s->d_jobs, 0, sizeof(Job) * n) != cudaSuccess) {
        cudaGetLastError();
        trees_server_destroy(s);
        return TREES_ERR_CUDA;
    }
    s->used.assign(n, 0);
    s->seg.assign(n, {0u, 0u});
    for (int32_t i = max_jobs - 1; i >= 0; --i) s->free_entries.push_back(i);
    s->free_seg[0] = (uint32_t)s->ctx->cap;
    *out = s;
    return TREES_OK;
}

extern "C" void trees_server_destroy(trees_server *s) {
    if (!s) return;
    if (s->d_jobs) cudaFree(s->d_jobs);
    if (s->d_stage) cudaFree(s->d_stage);
    if (s->d_joff) cudaFree(s->d_joff);
    if (s->d_entries) cudaFree(s->d_entries);
    if (s->d_done) cudaFree(s->d_done);
    if (s->d_bc) cudaFree(s->d_bc);
    if (s->h_stage) cudaFreeHost(s->h_stage);
    if (s->h_entries) cudaFreeHost(s->h_entries);
    if (s->h_done) cudaFreeHost(s->h_done);
    if (s->h_bc) cudaFreeHost(s->h_bc);
    if (s->ctx) trees_destroy(s->ctx);
    delete s;
}

extern "C" int trees_server_submit(trees_server *s, const trees_job_t *job, uint64_t seg_slots, uint64_t *id) {
    if (!s || !job) return TREES_ERR_INVALID_ARG;
    const uint64_t want = seg_slots ? seg_slots : job_slots(job, nullptr);
    if (want == 0 || want > 0xFFFFFFFFull) return TREES_ERR_INVALID_ARG;
    if (want > s->ctx->cap) return TREES_ERR_ADMISSION;
    Job probe;
    const int rc = make_job_record(job, 0u, 1u, 0u, &probe);
    if (rc) return rc;
    trees_server::Pending p;
    p.job = *job;
    p.slots = want;
    p.id = s->next_id++;
    s->queue.push_back(p);
    if (id) *id = p.id;
    return TREES_OK;
}

extern "C" int trees_server_step(trees_server *s, void *stream) {
    if (!s) return TREES_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // admission: in arrival order, while an entry and a segment are free
    uint32_t na = 0;
    while (!s->queue.empty() && !s->free_entries.empty()) {
        const trees_server::Pending &p = s->queue.front();
        uint32_t base = 0;
        if (!seg_alloc(s, (uint32_t)p.slots, &base)) break;
        const int32_t e = s->free_entries.back();
        s->free_entries.pop_back();
        make_job_record(&p.job, base, (uint32_t)p.slots, p.id, &s->h_stage[na]);
        s->h_entries[na] = (uint32_t)e;
        s->used[e] = 1;
        s->seg[e] = {base, (uint32_t)p.slots};
        s->hw = std::max(s->hw, (uint32_t)e + 1u);
        ++na;
        ++s->running;
        s->queue.pop_front();
    }
    if (na) {
        if (cudaMemcpyAsync(s->d_stage, s->h_stage, sizeof(Job) * na, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(s->d_entries, s->h_entries, sizeof(uint32_t) * na, cudaMemcpyHostToDevice, st) !=
                cudaSuccess)
            return TREES_ERR_CUDA;
        k_admit<<<std::min<uint32_t>(na, 1024u), 256, 0, st>>>(s->d_jobs, s->d_stage, s->d_entries, na);
        if (cudaGetLastError() != cudaSuccess) return TREES_ERR_CUDA;
    }
    if (s->running == 0) return TREES_OK;
    std::memset(s->h_bc, 0, sizeof(BatchCtl));
    s->h_bc->njobs = s->hw;
    s->h_bc->max_epochs = s->ctx->cfg.max_epochs;
    if (cudaMemcpyAsync(s->d_bc, s->h_bc, sizeof(BatchCtl), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return TREES_ERR_CUDA;
    int rc = launch_batch(s->ctx, s->d_bc, s->d_jobs, s->d_joff, s->d_done, (uint32_t)s->steps, st);
    if (rc) return rc;
    ++s->launches;
    if (cudaMemcpyAsync(s->h_bc, s->d_bc, sizeof(BatchCtl), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return TREES_ERR_CUDA;
    int err = 0;
    if (cudaMemcpy(&err, &s->ctx->ctl->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return TREES_ERR_CUDA;
    const uint32_t nd = s->h_bc->done_count;
    if (nd) {
        if (cudaMemcpyAsync(s->h_done, s->d_done, sizeof(BatchDone) * nd, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return TREES_ERR_CUDA;
        for (uint32_t i = 0; i < nd; ++i) {
            const BatchDone &d = s->h_done[i];
            trees_job_result_t r;
            fill_result(d, &r);
            s->finished.push_back(r);
            const int32_t e = (int32_t)d.job;
            if (e >= 0 && e < s->max_jobs && s->used[e]) {
                s->used[e] = 0;
                seg_free(s, s->seg[e].first, s->seg[e].second);
                s->free_entries.push_back(e);
                --s->running;
            }
        }
        while (s->hw > 0 && !s->used[s->hw - 1]) --s->hw;
    }
    return err;
}

extern "C" int trees_server_poll(trees_server *s, trees_job_result_t *out, int32_t cap, int32_t *n) {
    if (!s || !n || (cap > 0 && !out)) return TREES_ERR_INVALID_ARG;
    const int32_t m = std::min<int32_t>(cap, (int32_t)s->finished.size());
    for (int32_t i = 0; i < m; ++i) out[i] = s->finished[i];
    s->finished.erase(s->finished.begin(), s->finished.begin() + m);
    *n = m;
    return TREES_OK;
}

extern "C" int trees_server_stats(trees_server *s, int32_t *queued, int32_t *running, uint64_t *launches) {
    if (!s) return TREES_ERR_INVALID_ARG;
    if (queued) *queued = (int32_t)s->queue.size();
    if (running) *running = s->running;
    if (launches) *launches = s->launches;
    return TREES_OK;
}

extern "C" int trees_server_replay(trees_server *s, const trees_job_t *jobs, const uint64_t *seg_slots,
                                   const double *arrival_s, int32_t n, int32_t plain, double *latency_s,
                                   trees_job_result_t *results, void *stream) {
    if (!s || !jobs || !arrival_s || !latency_s || !results || n <= 0) return TREES_ERR_INVALID_ARG;
    using clk = std::chrono::steady_clock;
    const auto t0 = clk::now();
    auto elapsed = [&]() { return std::chrono::duration<double>(clk::now() - t0).count(); };
    auto wait_until = [&](double t) {
        while (elapsed() < t) {
            const double d = t - elapsed();
            if (d > 200e-6) std::this_thread::sleep_for(std::chrono::duration<double>(d - 100e-6));
        }
    };
    if (plain) {  // one job per launch, first come first served
        for (int32_t i = 0; i < n; ++i) {
            wait_until(arrival_s[i]);
            int rc = trees_run(s->ctx, &jobs[i], stream);
            if (rc) return rc;
            const int status = trees_sync(s->ctx);
            const double t = elapsed();
            trees_stats_t st;
            trees_stats(s->ctx, &st);
            uint64_t v = 0;
            trees_result(s->ctx, 0, &v);
            trees_job_result_t &r = results[i];
            std::memset(&r, 0, sizeof(r));
            r.id = (uint64_t)i;
            r.result = (jobs[i].program == TREES_PROG_FIB || jobs[i].program == TREES_PROG_NQUEENS) ? v : 0;
            r.tasks = st.tasks;
            r.joins = st.joins;
            r.maps = st.maps;
            r.ns = st.ns;
            r.epochs = (uint32_t)st.epochs;
            r.peak_slots = (uint32_t)st.peak_slots;
            r.status = status;
            latency_s[i] = t - arrival_s[i];
        }
        return TREES_OK;
    }
    std::vector<int32_t> index_of_id;
    const uint64_t id0 = s->next_id;
    int32_t next = 0, done = 0;
    std::vector<trees_job_result_t> got((size_t)std::max(1, s->max_jobs));
    while (done < n) {
        while (next < n && arrival_s[next] <= elapsed()) {
            uint64_t id = 0;
            const int rc = trees_server_submit(s, &jobs[next], seg_slots ? seg_slots[next] : 0, &id);
            if (rc) return rc;
            ++next;
        }
        int32_t q = 0, r = 0;
        trees_server_stats(s, &q, &r, nullptr);
        if (q + r == 0) {
            if (next < n) wait_until(arrival_s[next]);
            continue;
        }
        const int rc = trees_server_step(s, stream);
        if (rc) return rc;
        const double t = elapsed();
        int32_t m = 0;
        trees_server_poll(s, got.data(), (int32_t)got.size(), &m);
        for (int32_t k = 0; k < m; ++k) {
            const int64_t i = (int64_t)(got[k].id - id0);
            if (i < 0 || i >= n) continue;
            results[i] = got[k];
            results[i].id = (uint64_t)i;
            latency_s[i] = t - arrival_s[i];
            ++done;
        }
    }
    return TREES_OK;
}
