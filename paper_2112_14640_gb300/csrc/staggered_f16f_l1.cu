// staggered_f16f_l1.cu -- one instantiation of the staggered stencil (f16 vectors, layout 1, FP32 links); see staggered.cuh.
#include "staggered.cuh"

namespace dgb {
template int launch_staggered_v<__half, 1, float>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
}  // namespace dgb
