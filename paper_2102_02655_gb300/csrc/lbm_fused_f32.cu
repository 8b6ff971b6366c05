// Fused bulk kernels for FP32 storage: the instantiations of
// lbm_fused_impl.cuh for one storage type, in a translation unit of their own
// so that the storage types compile in parallel.
#include "lbm_fused_impl.cuh"

namespace cglbm {

template int launch_fused<float, float>(const StepArgs<float>&, int, cudaStream_t);
template int launch_fused_batch<float, float>(const StepArgs<float>*, const int4*, int, int*, int, int,
                                            cudaStream_t, int*);

}  // namespace cglbm
