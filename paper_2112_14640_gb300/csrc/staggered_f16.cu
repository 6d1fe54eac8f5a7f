// staggered_f16.cu -- F16 instantiations of the staggered stencil (see staggered.cuh).
#include "staggered.cuh"

namespace dgb {
template int launch_staggered_t<__half>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
}  // namespace dgb
