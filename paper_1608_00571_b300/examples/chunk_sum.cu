// A user task program for the TREES runtime (include/trees_program.cuh):
// the sum of n 32-bit keys as a task tree.  SUM(lo, hi) sums keys[lo, hi):
// a range of at most `chunk` keys is one map unit that a whole block
// reduces; a longer range forks k = min(arity, ceil(len / chunk)) children
// over equal parts (part i = [lo + len*i/k, lo + len*(i+1)/k)) and joins
// ADD, which adds the children's results.  Parameters: ptr[0] = the keys
// (device, u32), val[0] = chunk, val[1] = arity, val[2] = keys per map unit
// (0 = a leaf is one unit; otherwise a leaf emits 0 and its units add their
// partial sums to its result atomically).
#include "trees_program.cuh"

struct ChunkSum {
    static constexpr uint32_t SUM = 1, ADD = 2;

    __device__ static uint32_t parts(uint32_t lo, uint32_t hi, const trees_user_env &env) {
        const uint64_t len = hi - lo, chunk = env.val[0], arity = env.val[1];
        const uint64_t need = (len + chunk - 1) / chunk;
        return (uint32_t)(need < arity ? need : arity);
    }

    __device__ static trees_user_plan plan(const trees_user_task &t, const trees_user_env &env) {
        trees_user_plan q = {};
        if (t.type == SUM) {
            if ((uint64_t)(t.a1 - t.a0) <= env.val[0]) {
                const uint64_t upk = env.val[2], len = t.a1 - t.a0;
                if (t.a1 > t.a0) {  // one block per unit sums the chunk
                    trees_map(q, upk ? (uint32_t)((len + upk - 1) / upk) : 1u, t.a0, t.a1);
                    if (upk) trees_emit(q, 0);  // the units add into it
                } else {
                    trees_emit(q, 0);  // an empty range sums to 0
                }
            } else {
                trees_fork(q, parts(t.a0, t.a1, env));
            }
        } else {  // ADD: the children's results
            const uint32_t k = parts(t.a0, t.a1, env);
            uint64_t sum = 0;
            for (uint32_t i = 0; i < k; ++i) sum += env.result[t.link + i];
            trees_emit(q, sum);
        }
        return q;
    }

    __device__ static trees_user_child child(const trees_user_task &t, uint32_t i, const trees_user_env &env) {
        const uint32_t k = parts(t.a0, t.a1, env);
        const uint64_t len = t.a1 - t.a0;
        return trees_task(SUM, t.a0 + (uint32_t)(len * i / k), t.a0 + (uint32_t)(len * (i + 1) / k));
    }

    __device__ static trees_user_child join(const trees_user_task &t, const trees_user_env &) {
        return trees_join(ADD, t.a0, t.a1);
    }

    // One block sums keys[m.a, m.b): per-thread partial sums, a warp
    // reduction, then one word per warp through shared memory.
    template <int BS>
    __device__ static void map(const trees_user_map &m, uint32_t unit, const trees_user_env &env, void *smem) {
        const uint32_t *keys = static_cast<const uint32_t *>(env.ptr[0]);
        const uint64_t upk = env.val[2];
        const uint32_t lo = upk ? m.a + (uint32_t)(unit * upk) : m.a;
        const uint32_t hi = upk ? (uint32_t)min((uint64_t)m.b, lo + upk) : m.b;
        unsigned long long s = 0;
        for (uint32_t i = lo + threadIdx.x; i < hi; i += BS) s += keys[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        unsigned long long *red = static_cast<unsigned long long *>(smem);
        if ((threadIdx.x & 31u) == 0u) red[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long tot = 0;
            for (int w = 0; w < BS / 32; ++w) tot += red[w];
            if (upk) atomicAdd(reinterpret_cast<unsigned long long *>(env.result + m.slot), tot);
            else env.result[m.slot] = tot;
        }
    }
};

TREES_DEFINE_PROGRAM(trees_chunk_sum, ChunkSum)
