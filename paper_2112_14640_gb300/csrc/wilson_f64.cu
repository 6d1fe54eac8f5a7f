// wilson_f64.cu -- F64 instantiations of the wilson stencil (see wilson.cuh).
#include "wilson.cuh"

namespace dgb {
template int launch_wilson_t<double>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
}  // namespace dgb
