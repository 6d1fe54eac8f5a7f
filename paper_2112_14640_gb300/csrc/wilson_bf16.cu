// wilson_bf16.cu -- BF16 instantiations of the wilson stencil (see wilson.cuh).
#include "wilson.cuh"

namespace dgb {
template int launch_wilson_t<__nv_bfloat16>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
}  // namespace dgb
