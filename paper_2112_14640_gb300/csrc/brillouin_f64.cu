// brillouin_f64.cu -- F64 instantiations of the brillouin stencil (see brillouin.cuh).
#include "brillouin.cuh"

namespace dgb {
template int launch_brillouin_t<double>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
}  // namespace dgb
