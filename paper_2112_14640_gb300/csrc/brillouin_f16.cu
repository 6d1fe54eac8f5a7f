// brillouin_f16.cu -- F16 instantiations of the brillouin stencil (see brillouin.cuh).
#include "brillouin.cuh"

namespace dgb {
template int launch_brillouin_t<__half>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
}  // namespace dgb
