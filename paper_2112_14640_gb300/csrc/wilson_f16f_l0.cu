// wilson_f16f_l0.cu -- one instantiation of the wilson stencil (f16 vectors, layout 0, FP32 links); see wilson.cuh.
#include "wilson.cuh"

namespace dgb {
template int launch_wilson_v<__half, 0, float>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
}  // namespace dgb
