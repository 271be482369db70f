// pfo_kernels_f32.cu -- the persistent PFO kernel variants for f32 TSDF storage.
#include "pfo_kernel.cuh"

namespace rf {

PfoFn pfo_fn_f32(int mode, int group) { return pfo_fn_dtype<RF_F32>(mode, group); }

}  // namespace rf
