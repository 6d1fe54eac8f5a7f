// wilson_f32.cu -- F32 instantiations of the wilson stencil (see wilson.cuh).
#include "wilson.cuh"

namespace dgb {
template int launch_wilson_t<float>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
}  // namespace dgb
