// Batched and served task trees: many independent jobs share one persistent
// launch.  Each job owns a segment of the task vector and its own epoch
// state (CEN, range stack, nextFreeCore, counters).  A global step runs the
// current epoch of every live job: block 0 applies Phase 3 and Phase 1 of
// every job (Sec. 5.2.2, 5.2.4) and lays the jobs' ranges end to end (an
// exclusive scan of range sizes); then the whole grid runs Phase 2 over that
// concatenated work list, so critical-path overhead is paid once per step for
// all jobs (work-together Tenet 1, Sec. 3).  Forks are allocated per job with
// a warp-segmented scan and one atomic per job per warp.
//
// Included by trees.cu (one translation unit).
#pragma once

#include "trees_impl/trees_dev.cuh"
#include "trees_impl/trees_programs.cuh"

namespace trees {

constexpr int BSTK = 64;  // range-stack entries per batched job
constexpr uint32_t PM_BATCH = PM_FIB | PM_MS | PM_NQ | PM_TRAV;  // programs a batch may mix

enum JobState : int32_t { JOB_FREE = 0, JOB_NEW = 1, JOB_ACTIVE = 2, JOB_DONE = 3 };

struct Job {
    RunParams rp;
    uint32_t seg_base, seg_cap;  // global TV slots [seg_base, seg_base + seg_cap)
    uint32_t type0, a00, a10;    // root task
    int32_t state, err;
    uint32_t pending;            // a range was popped and ran: Phase 3 is due
    uint32_t sp, next, cen, lo, hi, base;
    uint32_t epochs, peak;
    unsigned int cnt, join;      // forks / joinScheduled of the job's current epoch
    unsigned long long tasks, joins, maps;
    unsigned long long t_admit;
    uint64_t id;
    Range stk[BSTK];
};

struct BatchDone {
    uint64_t id;
    uint32_t job;
    int32_t status;
    uint32_t epochs, peak;
    unsigned long long result, tasks, joins, maps, ns;
};

struct BatchCtl {
    unsigned int njobs;       // job-table entries Phase A scans
    unsigned int done_count;  // completion records appended since the host last read them
    unsigned int W;           // work items of the current step
    unsigned int active;      // jobs that ran in the current step
    unsigned int steps;       // steps executed by the last launch
    unsigned int max_epochs;
    unsigned int pad[2];
};

// Phase 3 of the epoch a job just ran, then Phase 1 of its next epoch.
// Returns the number of TV entries the job launches this step.
__device__ __forceinline__ uint32_t job_advance(const Conf &c, Job &J, uint32_t j, bool last_step, BatchCtl *bc,
                                                BatchDone *done) {
    if (J.state == JOB_NEW) {
        const uint32_t r = J.seg_base;
        c.code[r] = enc(0u, J.type0);
        c.a0[r] = J.a00;
        c.a1[r] = J.a10;
        c.link[r] = 0u;
        c.result[r] = 0ull;
        J.sp = 1;
        J.stk[0] = Range{0u, r, r + 1u, 0u};
        J.next = r + 1u;
        J.peak = 1u;
        J.pending = 0u;
        J.epochs = 0u;
        J.t_admit = globaltimer();
        J.state = JOB_ACTIVE;
    }
    if (J.state != JOB_ACTIVE) return 0u;
    if (J.pending) {
        const uint32_t f = vload(&J.cnt), jf = vload(&J.join);
        if (jf) {
            if (J.sp < BSTK) J.stk[J.sp++] = Range{J.cen, J.lo, J.hi, 1u};
            else J.err = TREES_ERR_STACK;
        }
        if (f) {
            if (J.sp < BSTK) J.stk[J.sp++] = Range{J.cen + 1u, J.base, J.base + f, 0u};
            else J.err = TREES_ERR_STACK;
            J.next = J.base + f;
            J.peak = max(J.peak, J.next - J.seg_base);
        } else if (!jf) {
            J.next = J.lo;  // neither forks nor joins: nextFreeCore decreases (Sec. 5.3)
        }
        J.epochs++;
        J.pending = 0u;
    }
    const int32_t err = vload(&J.err);
    const bool finished = err != 0 || J.sp == 0u;
    if (!finished && J.epochs >= bc->max_epochs) J.err = TREES_ERR_EPOCH_LIMIT;
    if (finished || J.err) {
        const uint32_t k = atomicAdd(&bc->done_count, 1u);
        BatchDone d;
        d.id = J.id;
        d.job = j;
        d.status = J.err;
        d.epochs = J.epochs;
        d.peak = J.peak;
        d.result = J.err ? 0ull : c.result[J.seg_base];
        d.tasks = J.tasks;
        d.joins = J.joins;
        d.maps = J.maps;
        d.ns = globaltimer() - J.t_admit;
        done[k] = d;
        J.state = JOB_DONE;
        return 0u;
    }
    if (last_step) return 0u;  // paused: resumes with Phase 1 at the next launch
    const Range r = J.stk[--J.sp];
    J.cen = r.cen;
    J.lo = r.lo;
    J.hi = r.hi;
    J.base = J.next;
    J.cnt = 0u;
    J.join = 0u;
    J.pending = 1u;
    return r.hi - r.lo;
}

// Phase A of a global step (block 0 only): advance every job and write the
// exclusive prefix of their range sizes into joff[0..njobs].
template <int BS>
__device__ void batch_phase_a(const Conf &c, Ctl *ctl, Smem<BS> &sm, BatchCtl *bc, Job *jobs, uint32_t *joff,
                              BatchDone *done, bool last_step) {
    const uint32_t nj = bc->njobs;
    const uint32_t per = (nj + BS - 1) / BS;
    const uint32_t j0 = threadIdx.x * per, j1 = min(j0 + per, nj);
    uint32_t sum = 0, act = 0;
    for (uint32_t j = j0; j < j1; ++j) {
        const uint32_t w = job_advance(c, jobs[j], j, last_step, bc, done);
        joff[j] = w;
        sum += w;
        act += w != 0u;
    }
    uint32_t total;
    int any;
    const uint32_t off = block_scan_u32<BS>(sum, act != 0u, &total, &any, sm);
    uint32_t run = off;
    for (uint32_t j = j0; j < j1; ++j) {
        const uint32_t w = joff[j];
        joff[j] = run;
        run += w;
    }
    if (threadIdx.x == 0) {
        joff[nj] = total;
        bc->W = total;
        ctl->mt_ctr[0] = 0ull;
        ctl->me_ctr[0] = 0ull;
    }
    __syncthreads();
}

__device__ __forceinline__ uint32_t find_job(const uint32_t *joff, uint32_t nj, uint32_t w) {
    uint32_t lo = 0, hi = nj;  // largest j with joff[j] <= w
    while (hi - lo > 1u) {
        const uint32_t mid = (lo + hi) >> 1;
        if (joff[mid] <= w) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Exclusive scan of x within runs of equal `key` across a warp (lanes are
// ordered by key).  Returns the exclusive prefix; *seg_end = last lane of the
// caller's run, *seg_total = the run's sum (valid on every lane).
__device__ __forceinline__ uint32_t warp_seg_scan(uint32_t key, uint32_t x, int *seg_end, uint32_t *seg_total) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t prev = __shfl_up_sync(0xffffffffu, key, 1);
    const bool head = lane == 0u || prev != key;
    const uint32_t heads = __ballot_sync(0xffffffffu, head);
    const uint32_t le = lane == 31u ? 0xffffffffu : ((2u << lane) - 1u);
    const int start = 31 - __clz(heads & le);
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if ((int)lane - o >= start) inc += y;
    }
    const uint32_t later = heads & ~le;
    const int end = later ? (__ffs(later) - 2) : 31;
    *seg_end = end;
    *seg_total = __shfl_sync(0xffffffffu, inc, end);
    return inc - x;
}

// largest j in [lo, hi) with joff[j] <= w
__device__ __forceinline__ uint32_t find_job_in(const uint32_t *joff, uint32_t lo, uint32_t hi, uint32_t w) {
    while (hi - lo > 1u) {
        const uint32_t mid = (lo + hi) >> 1;
        if (joff[mid] <= w) lo = mid;
        else hi = mid;
    }
    return lo;
}

// One Phase-2 tile of a global step: work items [t0, t0 + BS).  Thread 0
// finds the jobs of the tile's first and last items; a tile inside one job
// (the common case) allocates its forks with one block scan and one atomic,
// a tile that straddles jobs with a warp-segmented scan and one atomic per
// job per warp.
template <int BS>
__device__ void batch_tile(const Conf &c, Ctl *ctl, Smem<BS> &sm, Job *jobs, const uint32_t *joff, uint32_t nj,
                           unsigned long long t0, uint32_t W, Acc &acc) {
    const uint32_t NONE = 0xffffffffu;
    if (threadIdx.x == 0) {
        const uint32_t last = (uint32_t)min(t0 + (unsigned long long)BS, (unsigned long long)W) - 1u;
        const uint32_t jf = find_job(joff, nj, (uint32_t)t0);
        sm.bc32[0] = jf;
        sm.bc32[1] = find_job_in(joff, jf, nj, last);
    }
    __syncthreads();
    const uint32_t jf = sm.bc32[0], jl = sm.bc32[1];
    const bool uniform = jf == jl;
    const unsigned long long wl = t0 + threadIdx.x;
    const bool inr = wl < W;
    const uint32_t w = (uint32_t)wl;
    Plan p[1];
    p[0].s = 0u;
    p[0].t = 0u;
    p[0].n = 0u;
    p[0].m = 0u;
    p[0].a0 = p[0].a1 = 0u;
    uint32_t j = NONE, cen = 0u;
    Job *J = nullptr;
    if (inr) {
        j = uniform ? jf : find_job_in(joff, jf, jl + 1u, w);
        J = &jobs[j];
        cen = J->cen;
        const uint32_t s = J->lo + (w - joff[j]);
        p[0].s = s;
        const uint32_t t = task_type(c.code[s], cen);
        p[0].t = t;
        if (t) {
            acc.valid++;
            const uint32_t a0 = needs_a0(t) ? c.a0[s] : 0u, a1 = needs_a1(t) ? c.a1[s] : 0u;
            const uint32_t lk = needs_link(t) ? c.link[s] : 0u;
            plan_task<PM_BATCH, merge_tile(BS)>(c, J->rp, p[0], cen, J->epochs, a0, a1, lk);
        }
    }
    const uint32_t nfork = forks_of(p[0]);
    uint32_t joined = 0u;
    if (uniform) {
        Job *JU = &jobs[jf];
        uint32_t ftot;
        int any;
        const uint32_t foff = block_scan_u32<BS>(nfork, 0, &ftot, &any, sm);
        if (ftot) {
            if (threadIdx.x == 0) {
                const uint32_t b = atomicAdd(&JU->cnt, ftot);
                const bool over =
                    (unsigned long long)JU->base + b + ftot > (unsigned long long)JU->seg_base + JU->seg_cap;
                if (over) atomicCAS(&JU->err, 0, TREES_ERR_CAPACITY);
                sm.bc32[2] = b;
                sm.bc32[3] = over;
            }
            __syncthreads();
            if (nfork && !sm.bc32[3]) joined = commit_task<PM_BATCH>(c, JU->rp, p[0], cen, JU->base + sm.bc32[2] + foff);
        }
        const uint32_t vt = (uint32_t)__syncthreads_count(p[0].t != 0u);
        const uint32_t jt = (uint32_t)__syncthreads_count(joined != 0u);
        if (threadIdx.x == 0) {
            if (vt) atomicAdd(&JU->tasks, (unsigned long long)vt);
            if (jt) {
                atomicAdd(&JU->joins, (unsigned long long)jt);
                JU->join = 1u;
            }
        }
    } else {
        int end;
        uint32_t ftot;
        const uint32_t excl = warp_seg_scan(j, nfork, &end, &ftot);
        const uint32_t lane = threadIdx.x & 31u;
        uint32_t b = 0u, over = 0u;
        if ((int)lane == end && j != NONE && ftot) {
            b = atomicAdd(&J->cnt, ftot);
            if ((unsigned long long)J->base + b + ftot > (unsigned long long)J->seg_base + J->seg_cap) {
                over = 1u;
                atomicCAS(&J->err, 0, TREES_ERR_CAPACITY);
            }
        }
        b = __shfl_sync(0xffffffffu, b, end);
        over = __shfl_sync(0xffffffffu, over, end);
        if (nfork && !over) joined = commit_task<PM_BATCH>(c, J->rp, p[0], cen, J->base + b + excl);
        uint32_t vt, jt;
        warp_seg_scan(j, p[0].t != 0u, &end, &vt);
        warp_seg_scan(j, joined, &end, &jt);
        if ((int)lane == end && j != NONE) {
            if (vt) atomicAdd(&J->tasks, (unsigned long long)vt);
            if (jt) {
                atomicAdd(&J->joins, (unsigned long long)jt);
                J->join = 1u;
            }
        }
    }
    acc.joins += joined;
    if (p[0].m) atomicAdd(&J->maps, 1ull);
    if (__syncthreads_or(p[0].m != 0u)) map_alloc<BS, 1>(c, ctl, sm, p, cen, 0u, 0u, j, acc);
    __syncthreads();
}

template <int BS>
__global__ void __launch_bounds__(BS) k_batch(Ctl *ctl, Conf c, BatchCtl *bc, Job *jobs, uint32_t *joff,
                                              BatchDone *done, uint32_t max_steps, unsigned long long *blk) {
    __shared__ Smem<BS> sm;
    __shared__ uint32_t s_w;
    uint32_t bar = 0;
    Acc acc = {0u, 0u, 0u};
    uint32_t step = 0;
    for (;; ++step) {
        if (blockIdx.x == 0) batch_phase_a<BS>(c, ctl, sm, bc, jobs, joff, done, step >= max_steps);
        if (!grid_sync<BS>(ctl, &bar, c.timeout_ns, sm)) break;
        if (threadIdx.x == 0) s_w = vload(&bc->W);
        __syncthreads();
        const uint32_t W = s_w, nj = bc->njobs;
        if (W == 0u) break;
        for (unsigned long long t0 = (unsigned long long)blockIdx.x * BS; t0 < W; t0 += (unsigned long long)gridDim.x * BS)
            batch_tile<BS>(c, ctl, sm, jobs, joff, nj, t0, W, acc);
        if (!grid_sync<BS>(ctl, &bar, c.timeout_ns, sm)) break;
        const unsigned long long mt = vload(&ctl->mt_ctr[0]);
        if (mt) {
            if (needs_partition(mt)) {
                partition_phase<BS>(c, mt, &jobs[0].rp, (uint32_t)sizeof(Job));
                if (!grid_sync<BS>(ctl, &bar, c.timeout_ns, sm)) break;
            }
            map_phase<BS, PM_BATCH>(c, ctl, sm, 0u, step, 0u, 0u, mt, 0ull, &jobs[0].rp, (uint32_t)sizeof(Job));
            if (!grid_sync<BS>(ctl, &bar, c.timeout_ns, sm)) break;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) bc->steps = step;
    (void)blk;
}

// Copies freshly admitted job records into their table entries.
__global__ void k_admit(Job *jobs, const Job *staged, const uint32_t *entries, uint32_t n) {
    const uint32_t words = sizeof(Job) / 4;
    for (uint32_t i = blockIdx.x; i < n; i += gridDim.x) {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(staged + i);
        uint32_t *dst = reinterpret_cast<uint32_t *>(jobs + entries[i]);
        for (uint32_t k = threadIdx.x; k < words; k += blockDim.x) dst[k] = src[k];
    }
}

}  // namespace trees
