// wilson_f16_l1.cu -- one instantiation of the wilson stencil (f16 vectors, layout 1, f16 links); see wilson.cuh.
#include "wilson.cuh"

namespace dgb {
template int launch_wilson_v<__half, 1, __half>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
}  // namespace dgb
