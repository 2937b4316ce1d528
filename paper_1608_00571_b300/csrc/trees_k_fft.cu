// Persistent epoch-loop kernels for one program (PM_FFT), every block size
// and slots-per-thread setting.
#include "trees_impl/trees_kernels.cuh"

namespace trees {

const void *persistent_kernel_fft(int bs, int tpt) { return persistent_kernel_for<PM_FFT>(bs, tpt); }

}  // namespace trees
