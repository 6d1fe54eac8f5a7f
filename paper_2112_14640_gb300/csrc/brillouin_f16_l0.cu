// brillouin_f16_l0.cu -- one instantiation of the brillouin stencil (f16 vectors, layout 0, f16 links); see brillouin.cuh.
#include "brillouin.cuh"

namespace dgb {
template int launch_brillouin_v<__half, 0, __half>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
}  // namespace dgb
