// Persistent epoch-loop kernels for one program (PM_MS), every block size and
// slots-per-thread setting.
#include "trees_impl/trees_kernels.cuh"

namespace trees {

const void *persistent_kernel_ms(int bs, int tpt) { return persistent_kernel_for<PM_MS>(bs, tpt); }

}  // namespace trees
