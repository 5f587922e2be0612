// float instantiation of the solver kernels.
// FP32 stencil arithmetic; time steps, QoI sums and totals stay FP64.
#include "kernels.cuh"

namespace ofm {
namespace gpu {
template int set_smem_attrs<float>();
template int launch_step<float>(const Params<float>&, const Params<float>&, int, int, cudaStream_t, long long*);
template int launch_init<float>(const Params<float>&, cudaStream_t, bool, long long*);
template int launch_stage<float>(const Params<float>&, const Params<float>&, int, int, int, cudaStream_t, long long*);
template int launch_totals<float>(const Params<float>&, cudaStream_t, int, long long*);
}  // namespace gpu
}  // namespace ofm
