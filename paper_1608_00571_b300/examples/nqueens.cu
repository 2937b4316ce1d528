// A user task program for the TREES runtime (include/trees_program.cuh):
// N-Queens solution counting as a task tree (Sec. 6.5 names the program).
// A ROW task holds a partial placement of queens in rows 0..r-1: a0 = cols
// | r << 16, a1 = d1 | d2 << 16, with cols the occupied columns and d1, d2
// the columns attacked along the two diagonals in row r.  With r == n it
// emits 1 (a solution); with no safe column it emits 0; otherwise it forks
// one ROW child per safe column, lowest column first (a variable number of
// children), and joins SUM, which adds its children's counts.
// Parameters: val[0] = n (1..16).
#include "trees_program.cuh"

struct NQueens {
    static constexpr uint32_t ROW = 1, SUM = 2;

    // The columns of row r where a queen is safe.
    __device__ static uint32_t free_cols(uint32_t a0, uint32_t a1, uint32_t n) {
        return ~((a0 & 0xFFFFu) | (a1 & 0xFFFFu) | (a1 >> 16)) & ((1u << n) - 1u);
    }

    __device__ static trees_user_plan plan(const trees_user_task &t, const trees_user_env &env) {
        trees_user_plan q = {};
        const uint32_t n = (uint32_t)env.val[0];
        const uint32_t fr = free_cols(t.a0, t.a1, n);
        if (t.type == ROW) {
            if ((t.a0 >> 16) == n) trees_emit(q, 1);          // all n queens placed
            else if (fr == 0u) trees_emit(q, 0);              // dead end
            else trees_fork(q, (uint32_t)__popc(fr));         // one child per safe column
        } else {  // SUM: one count per child, in the order they were forked
            uint64_t s = 0;
            for (uint32_t i = 0; i < (uint32_t)__popc(fr); ++i) s += env.result[t.link + i];
            trees_emit(q, s);
        }
        return q;
    }

    // Child i: a queen on the i-th lowest safe column of row r.
    __device__ static trees_user_child child(const trees_user_task &t, uint32_t i, const trees_user_env &env) {
        const uint32_t n = (uint32_t)env.val[0], mask = (1u << n) - 1u;
        uint32_t fr = free_cols(t.a0, t.a1, n);
        for (uint32_t k = 0; k < i; ++k) fr &= fr - 1u;  // drop the i lowest safe columns
        const uint32_t b = fr & (0u - fr);
        const uint32_t r = t.a0 >> 16, cols = t.a0 & 0xFFFFu, d1 = t.a1 & 0xFFFFu, d2 = t.a1 >> 16;
        return trees_task(ROW, (cols | b) | ((r + 1u) << 16), (((d1 | b) << 1) & mask) | (((d2 | b) >> 1) << 16));
    }

    // The continuation keeps the row's arguments: SUM recounts its children from them.
    __device__ static trees_user_child join(const trees_user_task &t, const trees_user_env &) {
        return trees_join(SUM, t.a0, t.a1);
    }

    template <int BS>
    __device__ static void map(const trees_user_map &, uint32_t, const trees_user_env &, void *) {}  // no maps
};

TREES_DEFINE_PROGRAM(trees_nqueens_program, NQueens)
