/*
 * trees.h -- C ABI of libtrees, a B300 (sm_103a) implementation of the TREES
 * epoch step: the Task Vector Machine of Sec. 4 run by a GPU-resident
 * scheduler.  Every task in the current epoch runs in parallel (Sec. 4.3.2);
 * forks take task-vector slots through a cooperative block scan and one
 * atomic per block (Sec. 5.2.3); joins rewrite the task's own slot as a
 * continuation for a later epoch (Sec. 4.3.2); the whole GPU synchronises
 * once between epochs (work-together Tenet 1, Sec. 3).
 *
 * Conventions
 *  - Every call returns an int status: TREES_OK (0) or one TREES_ERR_* code.
 *    Device-side failures (a full task vector, an epoch limit, a barrier
 *    wait that ran out) are sticky flags that the run sets instead of
 *    trapping; trees_sync() returns them.
 *  - Pointers named dev_* / device pointers are CUDA device memory owned by
 *    the caller (e.g. a torch tensor's data_ptr()); host pointers are plain
 *    host memory.  The library never frees caller memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Runs are asynchronous and stream ordered; one context runs one
 *    job (or one batch) at a time, so calls on a context must be ordered on
 *    one stream or separated by trees_sync().
 *  - Capacities are counted in task-vector slots (one slot = one TV entry).
 */
#ifndef TREES_H
#define TREES_H

#include <stddef.h>
#include <stdint.h>

#include "trees_user.h"

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define TREES_OK 0
#define TREES_ERR_CAPACITY 1     /* a fork or map found the task vector / map list full */
#define TREES_ERR_EPOCH_LIMIT 2  /* the run reached config.max_epochs */
#define TREES_ERR_TIMEOUT 3      /* a grid barrier wait exceeded config.timeout_ns */
#define TREES_ERR_INVALID_ARG 4  /* bad argument; nothing was launched */
#define TREES_ERR_CUDA 5         /* a CUDA runtime call failed */
#define TREES_ERR_ADMISSION 6    /* serving: a job can never fit the configured memory */
#define TREES_ERR_STACK 7        /* the epoch-range stack overflowed */
#define TREES_ERR_BUSY 8         /* the context is still running a job */

/* ------------------------------------------------------------ task types
 * Sec. 5.1.2 footnote 2: a TV entry stores one integer, epoch*NTT + type,
 * with type in 1..NTT and 0 meaning "no task".  NTT = TREES_NUM_TASK_TYPES. */
#define TREES_TASK_FIB 1         /* fib(n): fork n-1, n-2, join FIB_SUM; leaf n<2 or n<=cutoff */
#define TREES_TASK_FIB_SUM 2     /* join: sum of the two children */
#define TREES_TASK_MS_SPLIT 3    /* mergesort split [lo,hi): leaf -> map leaf sort */
#define TREES_TASK_MS_MERGE 4    /* join: map merge of the two sorted halves */
#define TREES_TASK_NQ_ROW 5      /* N-Queens row: fork one child per safe column, join NQ_SUM */
#define TREES_TASK_NQ_SUM 6      /* join: sum of the children's counts */
#define TREES_TASK_BFS_VISIT 7   /* BFS vertex: map over its adjacency, claimed neighbours fork */
#define TREES_TASK_PO 8          /* postorder(node) of Fig. 2 */
#define TREES_TASK_PO_AFTER 9    /* visitAfter(node) of Fig. 2 (join) */
#define TREES_TASK_PRE 10        /* preorder(node) of Fig. 2 */
#define TREES_TASK_SSSP_RELAX 11 /* SSSP vertex (Sec. 6.3's worklist relaxation as tasks): map over its
                                    out-edges; a neighbour whose distance it shortens is forked once per epoch */
#define TREES_TASK_FFT 12        /* FFT (Sec. 6.2) of the points o, o + 2^d, o + 2*2^d, ... of the input:
                                    a leaf transforms them in its task, else it forks its even and odd points
                                    and joins FFT_COMBINE */
#define TREES_TASK_FFT_COMBINE 13 /* join: radix-2 butterflies merging the two half transforms, in the task
                                     or, above the cutoff, as a map over the butterflies */
#define TREES_NUM_TASK_TYPES 13

/* ------------------------------------------------------------ programs */
#define TREES_PROG_FIB 1
#define TREES_PROG_MERGESORT 2
#define TREES_PROG_NQUEENS 3
#define TREES_PROG_BFS 4
#define TREES_PROG_POSTORDER 5
#define TREES_PROG_PREORDER 6
#define TREES_PROG_SSSP 7
#define TREES_PROG_FFT 8
#define TREES_PROG_USER 9        /* a user task program (trees_program.cuh), run by its own kernel */

/* ------------------------------------------------------------ schedulers */
#define TREES_SCHED_PERSISTENT 0 /* one cooperative launch; one grid barrier per epoch */
#define TREES_SCHED_GRAPH 1      /* CUDA graph: epoch, map and Phase-3 kernels in a conditional WHILE node */
#define TREES_SCHED_HOSTLOOP 2   /* the paper's host loop: one launch and one device->host read per epoch (Sec. 5.2.4) */

typedef struct {
    int32_t block_size;      /* threads per block: 128, 256, 512 or 1024 (default 512) */
    int32_t blocks_per_sm;   /* persistent grid = SMs * this; 0 = as many as fit */
    int32_t scheduler;       /* TREES_SCHED_* */
    int32_t trace;           /* 1 = record the per-epoch trace (trees_trace) */
    uint32_t max_epochs;     /* 0 = 1<<20 */
    uint32_t trace_cap;      /* trace entries kept; 0 = 65536 */
    uint64_t timeout_ns;     /* grid-barrier wait limit; 0 = 2 s */
    uint64_t map_capacity;   /* map descriptors and map tiles per epoch; 0 = task-vector capacity */
    int32_t inject_stall_epoch; /* test hook, -1 = off: in that epoch the last block leaves
                                   without arriving at the barrier, so the others time out */
    int32_t grid_blocks;     /* persistent grid size; 0 = SMs * blocks_per_sm (capped at co-residency) */
    int32_t tasks_per_thread; /* TV slots a thread takes per Phase-2 tile: 1, 2 or 4 (0 = 2) */
    int32_t reserved;
} trees_config_t;

/* Fills *cfg with the defaults above.  The block size default follows the
 * work-group size of 256..512 work-items a TREES kernel is split into
 * (Sec. 5.1.1).  No error: a NULL cfg is ignored. */
void trees_default_config(trees_config_t *cfg);

/* ------------------------------------------------------------ context */
typedef struct trees_ctx trees_ctx;

/* Device bytes a context with `capacity_slots` TV slots needs (TV columns,
 * map lists, trace, control block): the Task Vector of Sec. 4 / 5.1.2 laid
 * out as a structure of arrays, 24 bytes per slot, plus the book-keeping
 * words of Sec. 5.1.2 (nextFreeCore, joinScheduled, mapScheduled) and the
 * epoch-range stack.  Returns 0 for invalid arguments. */
size_t trees_bytes_for(size_t capacity_slots, const trees_config_t *cfg);

/* Creates a context on the current CUDA device that owns a task vector of
 * capacity_slots entries (allocated with cudaMalloc): the Task Vector, Task
 * Mask Stack and book-keeping structures of Sec. 4 and Sec. 5.1.2, all in GPU
 * memory as Sec. 5.1.2 places them (the TMS as per-entry epoch numbers plus a
 * stack of NDRanges).  TV slot i is TVM core i (Sec. 5.1.1).  cfg may be NULL
 * (defaults).  capacity_slots must be in [1, 2^32-1].  *out receives the
 * context, owned by the caller until trees_destroy.  Errors: INVALID_ARG,
 * CUDA (allocation failed). */
int trees_create(size_t capacity_slots, const trees_config_t *cfg, trees_ctx **out);

/* Same structures (Sec. 5.1.2), but carved out of a caller-owned device
 * buffer of `bytes` bytes (256-byte aligned), e.g. a torch tensor; capacity
 * is the largest that fits.  The buffer must outlive the context and is never
 * freed by the library.  Errors: INVALID_ARG (NULL, unaligned or too small),
 * CUDA. */
int trees_create_on(void *dev_buf, size_t bytes, const trees_config_t *cfg, trees_ctx **out);

/* Releases the Task Vector and book-keeping structures the context
 * allocated (Sec. 5.1.2); never a caller buffer.  Call it once the context is
 * idle (after trees_sync).  NULL is ignored. */
void trees_destroy(trees_ctx *ctx);

/* Task-vector capacity of the context, in slots (TVM cores, Sec. 5.1.1). */
size_t trees_capacity(const trees_ctx *ctx);

/* Launch geometry the context uses: blocks in the persistent grid, threads
 * per block, SM count (the physical cores onto which Sec. 5.1.1 maps the
 * TVM's abstract cores).  Any output pointer may be NULL.  Errors:
 * INVALID_ARG (NULL context). */
int trees_geometry(const trees_ctx *ctx, int32_t *grid_blocks, int32_t *block_size, int32_t *sms);

/* ------------------------------------------------------------ one job */
/* A user task program compiled against trees_program.cuh by
 * TREES_DEFINE_PROGRAM: op TREES_USER_OP_OCCUPANCY writes to *out how many
 * blocks of block_size threads of its persistent kernel fit on one SM; op
 * TREES_USER_OP_LAUNCH launches that kernel cooperatively on `grid` blocks
 * with the kernel arguments `args` on `stream`.  Returns a cudaError_t value
 * (0 = success).  The program's kernels live in the caller's module; the
 * library calls this function instead of launching them itself. */
typedef int (*trees_program_fn)(int32_t op, int32_t block_size, int32_t tasks_per_thread, void **args, int32_t grid,
                                void *stream, int32_t *out);
#define TREES_USER_OP_OCCUPANCY 0
#define TREES_USER_OP_LAUNCH 1

typedef struct {
    int32_t program;          /* TREES_PROG_* */
    uint32_t n;               /* fib: n; N-Queens: board size (1..16); mergesort: number of keys;
                                 BFS, SSSP: source vertex; traversal: number of nodes;
                                 FFT: number of points, a power of two in [1, 2^25] */
    uint32_t cutoff;          /* fib: a call with n <= cutoff is a leaf computed in its task (0 = none);
                                 FFT: a combine of <= cutoff points runs in its task, a larger one as a
                                 map (0 = every combine is a map; >= n = none is, as in Sec. 6.2) */
    uint32_t leaf;            /* mergesort: leaf size, 1..1024 (0 = 1024);
                                 FFT: leaf transform size, 1, 2, 4, 8 or 16 (0 = 16) */
    uint32_t *keys;           /* mergesort: device keys, sorted in place */
    uint32_t *scratch;        /* mergesort: device buffer of n keys (NULL = the context's own) */
    const int32_t *row_ptr;   /* BFS, SSSP: device CSR row offsets [nv+1] */
    const int32_t *col;       /* BFS, SSSP: device CSR columns */
    int32_t *level;           /* BFS: device output [nv], -1 = unreachable */
    int32_t nv;               /* BFS, SSSP: vertex count */
    const int32_t *left;      /* traversal: device child arrays [n], -1 = nil; node 0 is the root */
    const int32_t *right;
    int32_t *visit_epoch;     /* traversal: device output [n], index of the epoch that visited the node */
    const uint32_t *weight;   /* SSSP: device edge weights aligned with col */
    uint64_t *dist;           /* SSSP: device output [nv], shortest distance from the source,
                                 UINT64_MAX = unreachable */
    uint32_t *sched;          /* SSSP: device scratch [nv]: the last epoch each vertex was forked for */
    const float *fft_in;      /* FFT: device input, n complex points as interleaved (re, im) fp32,
                                 8-byte aligned; read only */
    float *fft_out;           /* FFT: device output [2n] floats, X[k] = sum_j x[j] exp(-2 pi i j k / n);
                                 8-byte aligned, must not overlap fft_in */
    trees_program_fn user_program;  /* user program: its launcher (persistent scheduler only) */
    uint32_t user_type, user_a0, user_a1;  /* user program: the root task, type 1..TREES_NUM_TASK_TYPES */
    uint32_t user_pad;
    void *user_ptr[TREES_USER_PARAMS];     /* user program: parameters passed to its device functions */
    uint64_t user_val[TREES_USER_PARAMS];
} trees_job_t;

/* Sec. 5.2.1 initialisation + the epoch loop: writes the job's root task
 * into TV entry 0 for epoch 0 and runs epochs until the range stack is empty.
 * Asynchronous on `stream` for the persistent and graph schedulers; the host
 * loop scheduler returns when the run is over.  A TREES_PROG_USER job runs
 * its program's own persistent kernel (user_program; the graph and host-loop
 * schedulers, whose kernels are compiled for the built-in programs, reject
 * it).  Errors before launch: INVALID_ARG (bad job), BUSY, CUDA. */
int trees_run(trees_ctx *ctx, const trees_job_t *job, void *stream);

/* Waits for the context's last run and returns its status (TREES_OK or the
 * first device-side error).  This is the end of the run Sec. 5.2.4 detects
 * when the NDRange stack is empty after Phase 3; the status words are the
 * sticky flags the run sets instead of trapping. */
int trees_sync(trees_ctx *ctx);

/* Reads the result word of a TV slot after trees_sync: the value an `emit`
 * stored in the task's own entry (Sec. 4.2, 4.3.2); slot 0 holds the root
 * task's, e.g. fib(n) or the N-Queens count, since the root sits in TV entry 0
 * (Sec. 5.2.1).  *out is host memory.  Errors: INVALID_ARG (NULL, or slot
 * beyond the capacity), CUDA. */
int trees_result(trees_ctx *ctx, uint32_t slot, uint64_t *out);

typedef struct {
    uint64_t epochs;        /* epochs executed (Sec. 4.4.1: the critical path) */
    uint64_t tasks;         /* valid task executions, joins included (the work) */
    uint64_t forks;         /* TV slots handed out by forks */
    uint64_t joins;         /* join operations */
    uint64_t maps;          /* map operations */
    uint64_t peak_slots;    /* highest nextFreeCore reached */
    uint64_t final_slots;   /* nextFreeCore at halt (0 = the TV emptied, Sec. 5.3) */
    uint64_t ns;            /* device time of the epoch loop (globaltimer) */
    int32_t status;         /* TREES_OK or the device-side error */
    int32_t error_epoch;    /* epoch in which the error was raised */
    int32_t grid_blocks;    /* blocks of the run's grid */
    int32_t block_size;     /* threads per block */
} trees_stats_t;

/* Statistics of the last run (call after trees_sync). */
int trees_stats(trees_ctx *ctx, trees_stats_t *out);

typedef struct {
    uint32_t cen;     /* current epoch number (the popped join-stack value) */
    uint32_t lo, hi;  /* NDRange [lo, hi) launched */
    uint32_t valid;   /* entries whose code matched CEN */
    uint32_t forks;   /* nextFreeCore - oldNextFreeCore */
    uint32_t joined;  /* joinScheduled */
    uint32_t maps;    /* map operations scheduled */
    uint32_t ns_phase2;    /* persistent scheduler: ns from the previous epoch's end to the
                            * barrier after Phase 2 (0 under the other schedulers) */
    uint64_t t_ns;         /* globaltimer at the end of the epoch */
    uint32_t ns_partition; /* persistent scheduler: ns of the merge partition sub-phase */
    uint32_t ns_map;       /* persistent scheduler: ns of the map operations */
} trees_epoch_t;

/* Copies up to `cap` per-epoch records of the last run (config.trace = 1)
 * into host memory `out`; *n receives the number copied. */
int trees_trace(trees_ctx *ctx, trees_epoch_t *out, size_t cap, size_t *n);

/* Convenience forms of trees_run. */
int trees_fib(trees_ctx *ctx, uint32_t n, uint32_t cutoff, void *stream);
int trees_nqueens(trees_ctx *ctx, uint32_t n, void *stream);
int trees_mergesort_u32(trees_ctx *ctx, uint32_t *dev_keys, uint32_t *dev_scratch, uint32_t n, void *stream);
int trees_bfs(trees_ctx *ctx, const int32_t *dev_row_ptr, const int32_t *dev_col, int32_t nv, int32_t src,
              int32_t *dev_level, void *stream);
/* Single-source shortest paths as tasks (Sec. 6.3): relax(v) maps over v's
 * out-edges (dist[u] = min(dist[u], dist[v] + w) by atomic minimum) and forks
 * relax(u) for the next epoch for every u it shortened, once per epoch per
 * vertex (dev_sched dedupes); the run ends when an epoch shortens nothing.
 * Distances are u64 (no overflow for u32 weights); the task and epoch counts
 * depend on the order of the races, the distances do not.  Every task slot
 * stays in use until the run ends (no joins), so the context needs one slot
 * per relax task (at least the reachable vertices, more when vertices are
 * shortened again).  Errors: INVALID_ARG (null arrays, nv < 1, src out of
 * range), CAPACITY at run time. */
int trees_sssp(trees_ctx *ctx, const int32_t *dev_row_ptr, const int32_t *dev_col, const uint32_t *dev_weight,
               int32_t nv, int32_t src, uint64_t *dev_dist, uint32_t *dev_sched, void *stream);
/* Fast Fourier transform as tasks (Sec. 6.2, Fig. 6): the n-point DFT
 * X[k] = sum_j x[j] exp(-2 pi i j k / n) by radix-2 decimation in time.
 * FFT(o, d) transforms the n >> d points of index o modulo 2^d: at most
 * `leaf` points are transformed inside the task (registers), more fork the
 * even- and odd-numbered points and join a combine of n >> d points, run
 * inside its task when it is at most `cutoff` points, else as a map whose
 * butterflies the whole grid shares (the paper's FFT uses no maps; cutoff
 * >= n reproduces that).  dev_in and dev_out hold n complex fp32 values as
 * interleaved (re, im) pairs, 8-byte aligned, and must not overlap; dev_in
 * is not written.  Arithmetic is fp32: every butterfly computes
 * t = w * O[k] with fused multiply-adds in a fixed order and E[k] +- t,
 * w = exp(-2 pi i k / m) from sincospif on the exact quotient 2k/m, so the
 * output does not depend on leaf, cutoff, block size or scheduler.  Needs
 * 2^(D+1) - 1 task slots and 2^(D-1) map descriptors, D = log2(n / leaf).
 * Errors: INVALID_ARG (n not a power of two in [1, 2^25], leaf not a power
 * of two <= 16, null or misaligned or overlapping buffers), CAPACITY at run
 * time. */
int trees_fft(trees_ctx *ctx, const float *dev_in, float *dev_out, uint32_t n, uint32_t leaf, uint32_t cutoff,
              void *stream);

/* ------------------------------------------------------------ measurement */

/* The critical-path floor: a persistent kernel that does nothing but `iters`
 * of the scheduler's grid barrier, on the grid of the context's last
 * persistent run (else the context's default grid).  Writes the device time
 * per barrier in microseconds. */
int trees_barrier_floor(trees_ctx *ctx, uint32_t iters, void *stream, double *us_per_barrier);

/* ------------------------------------------------------------ autotuning */
typedef struct {
    trees_config_t cfg;  /* the candidate configuration */
    double ms;           /* its best time over the timed runs (device, CUDA events) */
    int32_t status;      /* TREES_OK, or why the candidate could not run */
    int32_t pad;
} trees_tune_entry_t;

/* Picks the configuration that runs `job` fastest on the current device:
 * every block size {128, 256, 512, 1024} x slots per thread {1, 2, 4} x scheduler
 * {persistent grid barrier, CUDA-graph relaunch}, each on a fresh context of
 * capacity_slots slots built from `base` (NULL = defaults), one warm-up and
 * `reps` timed runs.  A mergesort job's keys are restored from a copy before
 * every run.  With cache_path and key non-NULL the choice is looked up in and
 * written to a JSON file mapping keys to configurations (a cached key costs
 * no runs).  *best receives the configuration, *best_ms its time; up to
 * table_cap candidates are reported in table (may be NULL), *table_n how many.
 * Errors: INVALID_ARG, CUDA, or the job's own status when every candidate
 * fails. */
int trees_autotune(const trees_job_t *job, size_t capacity_slots, const trees_config_t *base, int32_t reps,
                   const char *cache_path, const char *key, trees_config_t *best, double *best_ms,
                   trees_tune_entry_t *table, int32_t table_cap, int32_t *table_n);

/* ------------------------------------------------------------ batches and serving
 * Many independent task trees share one persistent launch (work-together
 * Tenet 1, Sec. 3, applied across jobs): each job owns a segment of the task
 * vector and its own epoch state; a global step runs the current epoch of
 * every live job.  Batched jobs may be fib, N-Queens, mergesort (caller
 * scratch required) or a traversal; BFS runs only through trees_run. */
typedef struct {
    uint64_t id;            /* job index (batch) or submission id (server) */
    uint64_t result;        /* the root's emitted value (fib, N-Queens); 0 otherwise */
    uint64_t tasks;         /* valid task executions of this job */
    uint64_t joins;
    uint64_t maps;
    uint64_t ns;            /* device time from admission to completion */
    uint32_t epochs;        /* this job's epochs */
    uint32_t peak_slots;    /* highest slot used in its segment, + 1 */
    int32_t status;         /* TREES_OK or the job's own error (CAPACITY when its segment was too small) */
    int32_t pad;
} trees_job_result_t;

/* Task-vector slots a job needs at its peak.  *exact (may be NULL) is set to
 * 1 when the count is exact (fib, mergesort, traversal upper bound, BFS,
 * FFT: 2^(D+1) - 1 for D = log2(n / leaf)) and 0 when it is an estimate
 * (N-Queens: the backtracking tree is not known before it is explored; SSSP:
 * one slot per relax task, at least the vertex count, more when distances
 * drop again; a job that outgrows it ends with CAPACITY).  A user program's
 * tree is unknown to the library: 0 slots, not exact (size its context from
 * the program). */
uint64_t trees_job_slots(const trees_job_t *job, int32_t *exact);

/* Runs njobs jobs in one persistent launch on the context's task vector.
 * seg_slots[i] (host array; NULL = trees_job_slots) reserves each job's
 * segment; their sum must fit the context (else ADMISSION).  Asynchronous on
 * `stream`.  Errors before launch: INVALID_ARG (a job that cannot be batched),
 * ADMISSION, CUDA. */
int trees_batch_run(trees_ctx *ctx, const trees_job_t *jobs, const uint64_t *seg_slots, int32_t njobs, void *stream);

/* Waits for the batch and copies one record per job into out[0..njobs)
 * (host memory), in job order; *steps (may be NULL) receives the number of
 * global steps.  Returns the batch-wide status (TIMEOUT, CUDA) or TREES_OK;
 * per-job errors are in out[i].status. */
int trees_batch_results(trees_ctx *ctx, trees_job_result_t *out, int32_t njobs, uint32_t *steps);

typedef struct trees_server trees_server;

/* A continuous-batching server on the current device: a task-vector pool of
 * pool_slots slots, up to max_jobs jobs resident at once, and launches of at
 * most steps_per_launch global steps.  Job state stays on the device between
 * launches; jobs that arrive while others run are admitted at the next
 * launch when a table entry and a segment of their size are free (first
 * fit, in arrival order). */
int trees_server_create(size_t pool_slots, int32_t max_jobs, int32_t steps_per_launch, const trees_config_t *cfg,
                        trees_server **out);
void trees_server_destroy(trees_server *srv);

/* Queues a job (host call, no device work).  seg_slots = 0 uses
 * trees_job_slots.  ADMISSION if the job can never fit the pool. */
int trees_server_submit(trees_server *srv, const trees_job_t *job, uint64_t seg_slots, uint64_t *id);

/* Admits queued jobs, runs one launch and collects the jobs that finished.
 * Synchronous (returns when the launch is over). */
int trees_server_step(trees_server *srv, void *stream);

/* Moves up to cap finished jobs into out (host); *n receives how many. */
int trees_server_poll(trees_server *srv, trees_job_result_t *out, int32_t cap, int32_t *n);

/* Jobs waiting for admission, jobs resident on the device, launches so far. */
int trees_server_stats(trees_server *srv, int32_t *queued, int32_t *running, uint64_t *launches);

/* Replays a trace in real time: job i arrives arrival_s[i] seconds after the
 * start (non-decreasing).  plain = 0 serves through the continuous batch;
 * plain = 1 runs one job per launch in arrival order (trees_run).  Writes each
 * job's latency (completion - arrival, seconds) and record.  seg_slots may be
 * NULL.  Returns TREES_OK or the first launch-level error. */
int trees_server_replay(trees_server *srv, const trees_job_t *jobs, const uint64_t *seg_slots,
                        const double *arrival_s, int32_t n, int32_t plain, double *latency_s,
                        trees_job_result_t *results, void *stream);

/* ------------------------------------------------------------ allocation-free entry point
 * The paper has no counterpart to this call; it exists for callers that may
 * not allocate device memory when they run a job: code recorded into a CUDA
 * stream capture that must not allocate, hosts whose GPU memory budget is
 * fixed at start-up, and plug-ins whose host application owns the allocator.
 *
 * trees_fib_noalloc runs fib(n) (leaf when n < 2 or n <= cutoff) with the
 * persistent scheduler, with its task vector, control block and statistics
 * in one static device array of 26 MiB that is part of the library (every GPU
 * that loads libtrees holds it until the process exits).  It calls no
 * cudaMalloc, cudaFree or other allocating routine.
 *  - Limit: 1,048,576 task-vector slots, i.e. trees of at most that many
 *    tasks at their peak (fib(n) needs 2F(n+1)-1: n <= 28 without cutoff).
 *    Larger jobs return TREES_ERR_CAPACITY before anything is launched.
 *  - Outputs: *dev_result (device uint64) receives fib(n); *dev_status
 *    (device int32) receives TREES_OK or the run's device-side error.  Both
 *    are written asynchronously on `stream`.
 *  - The first call on a device looks up the array's device address and the
 *    launch geometry for that device (the device must be current); make that
 *    first call before any stream capture.
 *  - All calls share the array and it keeps the previous call's contents (the
 *    control block is cleared at each call).  Calls whose GPU work overlaps
 *    race on it: order them on one stream or with events.
 * Errors: INVALID_ARG (null output, n > 93, cutoff > 30), CAPACITY, CUDA. */
int trees_fib_noalloc(uint32_t n, uint32_t cutoff, uint64_t *dev_result, int32_t *dev_status, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* TREES_H */
