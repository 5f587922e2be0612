// double instantiation of the solver kernels.
// Compiled with -fmad=false: together with the operation order in
// kernels.cuh this makes the FP64 path round exactly as the FP64 reference.
#include "kernels.cuh"

namespace ofm {
namespace gpu {
template int set_smem_attrs<double>();
template int launch_step<double>(const Params<double>&, const Params<double>&, int, int, cudaStream_t, long long*);
template int launch_init<double>(const Params<double>&, cudaStream_t, bool, long long*);
template int launch_stage<double>(const Params<double>&, const Params<double>&, int, int, int, cudaStream_t, long long*);
template int launch_totals<double>(const Params<double>&, cudaStream_t, int, long long*);
}  // namespace gpu
}  // namespace ofm
