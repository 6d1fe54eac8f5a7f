// staggered_f32_l1.cu -- one instantiation of the staggered stencil (f32 vectors, layout 1, f32 links); see staggered.cuh.
#include "staggered.cuh"

namespace dgb {
template int launch_staggered_v<float, 1, float>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
}  // namespace dgb
