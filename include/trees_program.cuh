/*
 * trees_program.cuh -- writing a task program for the TREES runtime.
 *
 * The built-in programs (fib, mergesort, N-Queens, BFS, SSSP, traversals,
 * FFT) are compiled into libtrees.  A user program is a struct of four
 * device functions compiled by the user, with nvcc for sm_103a and this
 * directory alone on the include path (the engine's device code is in
 * trees_impl/), into the user's own shared library (for example
 *   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -std=c++17 -shared
 *        -Xcompiler -fPIC -I include prog.cu -o libprog.so);
 * TREES_DEFINE_PROGRAM(name, Prog) instantiates
 * the runtime's persistent epoch kernel for it (the persistent scheduler:
 * one grid barrier per epoch) and exports `name` with the trees_program_fn
 * signature of trees.h.  A job with program = TREES_PROG_USER, user_program
 * = that function, a root task (user_type, user_a0, user_a1) and up to four
 * pointers and values runs through trees_run like any other program; the
 * library sizes the grid and launches through the function, so the kernel
 * never leaves the user's module.
 *
 * The task model is the paper's (Sec. 4.1-4.3): a task of type
 * 1..TREES_NUM_TASK_TYPES with two 32-bit arguments runs in the epoch its
 * parent forked it for.  The runtime asks, for each task:
 *
 *   static __device__ trees_user_plan plan(const trees_user_task &t, const trees_user_env &env);
 *       What the task does: emit (result[t.slot] = value), fork `forks`
 *       children (arbitrary arity), or schedule a map of `map_units` units.
 *       A task that forks nothing (and maps or emits) ends.
 *   static __device__ trees_user_child child(const trees_user_task &t, uint32_t i, const trees_user_env &env);
 *       Child i < forks (type and arguments); children occupy consecutive
 *       slots in this order, the first at the continuation's t.link.  A
 *       child whose type is outside 1..TREES_NUM_TASK_TYPES never runs (its
 *       slot is left empty and its result word is not written).
 *   static __device__ trees_user_child join(const trees_user_task &t, const trees_user_env &env);
 *       The continuation the task turns into after forking (Sec. 4.3.2:
 *       its own slot, same epoch number, run after every task forked under
 *       it has finished); type 0 = none.  It reads its children's results
 *       at env.result[t.link + i].
 *   template <int BS> static __device__ void map(const trees_user_map &m, uint32_t unit,
 *                                                const trees_user_env &env, void *smem);
 *       One unit of a map, run by all BS threads of a block (so it may use
 *       __syncthreads()) with TREES_USER_SMEM_BYTES of shared memory at
 *       smem; the units of every map an epoch scheduled run after its tasks
 *       and before the next epoch (Sec. 5.2.4).
 *
 * plan runs in every thread that holds a task; child and join in the thread
 * that forked.  They must not synchronise: only map is block-cooperative.
 * A task that both forks and maps is treated as mapping (its forks are
 * dropped); emitting and mapping together is allowed, the map running after
 * the emit.  Size the context for the program: task-vector slots for its
 * widest set of live tasks, and map_capacity (trees_config_t) for the map
 * units of one epoch.
 */
#pragma once

#include "trees.h"
#include "trees_impl/trees_kernels.cuh"

// The paper's four primitives (Sec. 4.2) as helpers for the records above:
// plan fills a trees_user_plan with trees_emit / trees_fork / trees_map, and
// child and join return trees_join's or a child's (type, a0, a1) record.
//   emit v          -> trees_emit(q, v)
//   fork f(args) xk -> trees_fork(q, k) in plan; child(t, i) returns trees_task(f, args of child i)
//   join f(args)    -> join(t) returns trees_join(f, args)
//   map f(args)     -> trees_map(q, units, a, b); the program's map runs each unit
__device__ __forceinline__ void trees_emit(trees_user_plan &q, uint64_t v) {
    q.emit = 1;
    q.value = v;
}
__device__ __forceinline__ void trees_fork(trees_user_plan &q, uint32_t children) { q.forks = children; }
__device__ __forceinline__ void trees_map(trees_user_plan &q, uint32_t units, uint32_t a, uint32_t b) {
    q.map_units = units;
    q.map_a = a;
    q.map_b = b;
}
__device__ __forceinline__ trees_user_child trees_task(uint32_t type, uint32_t a0, uint32_t a1) {
    trees_user_child c;
    c.type = type;
    c.a0 = a0;
    c.a1 = a1;
    return c;
}
__device__ __forceinline__ trees_user_child trees_join(uint32_t type, uint32_t a0, uint32_t a1) {
    return trees_task(type, a0, a1);
}

#define TREES_DEFINE_PROGRAM(NAME, PROG)                                                                       \
    extern "C" int NAME(int32_t op, int32_t bs, int32_t tpt, void **args, int32_t grid, void *stream,         \
                        int32_t *out) {                                                                        \
        const void *k = trees::persistent_kernel_for<trees::PM_USER, PROG>(bs, tpt);                           \
        if (!k) return (int)cudaErrorInvalidValue;                                                             \
        if (op == TREES_USER_OP_OCCUPANCY) {                                                                   \
            int occ = 0;                                                                                       \
            const cudaError_t r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, bs, 0);               \
            if (out) *out = occ;                                                                               \
            return (int)r;                                                                                     \
        }                                                                                                      \
        if (op == TREES_USER_OP_LAUNCH)                                                                        \
            return (int)cudaLaunchCooperativeKernel(k, dim3(grid), dim3(bs), args, 0, (cudaStream_t)stream);   \
        return (int)cudaErrorInvalidValue;                                                                     \
    }
