// pfo_kernels_f16.cu -- the persistent PFO kernel variants for f16 TSDF storage.
#include "pfo_kernel.cuh"

namespace rf {

PfoFn pfo_fn_f16(int mode, int group) { return pfo_fn_dtype<RF_F16>(mode, group); }

}  // namespace rf
