/*
 * TREES user task programs: the records a user program's device functions
 * receive and return (C layout).  The device-side contract and the macro
 * that compiles a program into its persistent kernel are in
 * trees_program.cuh; trees.h's trees_job_t carries the program's launcher
 * (trees_program_fn), its root task and its parameters.
 *
 * A program is the paper's task model (Sec. 4.1-4.2): a task of type
 * 1..TREES_NUM_TASK_TYPES with two 32-bit arguments either emits a value
 * (its slot's result), forks children for the next epoch and turns into a
 * join continuation that runs once they have all finished (it finds them at
 * `link`, link + 1, ...), or schedules a map: data-parallel work of `units`
 * units, each run by a whole thread block, before the next epoch
 * (Sec. 4.2, 5.2.4).
 */
#ifndef TREES_USER_H
#define TREES_USER_H

#include <stdint.h>

#define TREES_USER_PARAMS 4          /* user pointers and values per job */
#define TREES_USER_SMEM_BYTES 32768  /* shared memory a block's map units may use */

/* The running task. */
typedef struct {
    uint32_t slot;  /* its task-vector entry (its result is result[slot]) */
    uint32_t type;  /* 1..TREES_NUM_TASK_TYPES */
    uint32_t a0, a1;
    uint32_t link;  /* a join continuation: the slot of its first child */
    uint32_t cen;   /* the epoch number it runs in */
} trees_user_task;

/* What a task does (returned by the program's plan). */
typedef struct {
    uint32_t forks;      /* children to fork (0 = none); then child() and join() are asked */
    uint32_t map_units;  /* > 0: schedule a map of this many units (a task that maps does not fork) */
    uint32_t map_a, map_b;
    int32_t emit;        /* nonzero: result[slot] = value */
    uint32_t pad;
    uint64_t value;
} trees_user_plan;

/* A forked child, or the join continuation (type 0 = the task ends instead). */
typedef struct {
    uint32_t type, a0, a1;
} trees_user_child;

/* A map scheduled by a task. */
typedef struct {
    uint32_t a, b;   /* the plan's map_a, map_b */
    uint32_t slot;   /* the scheduling task's slot */
    uint32_t units;  /* units of the map */
} trees_user_map;

/* The job's parameters and the result column. */
typedef struct {
    void *ptr[TREES_USER_PARAMS];
    uint64_t val[TREES_USER_PARAMS];
    uint64_t *result;  /* result[slot], one 64-bit word per task-vector entry */
} trees_user_env;

#endif
