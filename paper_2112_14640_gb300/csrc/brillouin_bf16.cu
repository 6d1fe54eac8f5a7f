// brillouin_bf16.cu -- BF16 instantiations of the brillouin stencil (see brillouin.cuh).
#include "brillouin.cuh"

namespace dgb {
template int launch_brillouin_t<__nv_bfloat16>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
}  // namespace dgb
