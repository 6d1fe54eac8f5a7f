// wilson_f32_l0.cu -- one instantiation of the wilson stencil (f32 vectors, layout 0, f32 links); see wilson.cuh.
#include "wilson.cuh"

namespace dgb {
template int launch_wilson_v<float, 0, float>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
}  // namespace dgb
