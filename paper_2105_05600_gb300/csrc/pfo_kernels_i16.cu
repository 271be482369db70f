// pfo_kernels_i16.cu -- the persistent PFO kernel variants for i16 TSDF storage.
#include "pfo_kernel.cuh"

namespace rf {

PfoFn pfo_fn_i16(int mode, int group) { return pfo_fn_dtype<RF_I16>(mode, group); }

}  // namespace rf
