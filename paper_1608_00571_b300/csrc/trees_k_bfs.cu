// Persistent epoch-loop kernels for one program (PM_BFS), every block size and
// slots-per-thread setting.
#include "trees_impl/trees_kernels.cuh"

namespace trees {

const void *persistent_kernel_bfs(int bs, int tpt) { return persistent_kernel_for<PM_BFS>(bs, tpt); }

}  // namespace trees
