// staggered_bf16.cu -- BF16 instantiations of the staggered stencil (see staggered.cuh).
#include "staggered.cuh"

namespace dgb {
template int launch_staggered_t<__nv_bfloat16>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
}  // namespace dgb
