// brillouin_bf16_l1.cu -- one instantiation of the brillouin stencil (bf16 vectors, layout 1, bf16 links); see brillouin.cuh.
#include "brillouin.cuh"

namespace dgb {
template int launch_brillouin_v<__nv_bfloat16, 1, __nv_bfloat16>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
}  // namespace dgb
