// staggered_bf16_l0.cu -- one instantiation of the staggered stencil (bf16 vectors, layout 0, bf16 links); see staggered.cuh.
#include "staggered.cuh"

namespace dgb {
template int launch_staggered_v<__nv_bfloat16, 0, __nv_bfloat16>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
}  // namespace dgb
