// staggered_f32.cu -- F32 instantiations of the staggered stencil (see staggered.cuh).
#include "staggered.cuh"

namespace dgb {
template int launch_staggered_t<float>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
}  // namespace dgb
