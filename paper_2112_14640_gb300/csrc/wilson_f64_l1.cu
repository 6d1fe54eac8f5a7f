// wilson_f64_l1.cu -- one instantiation of the wilson stencil (f64 vectors, layout 1, f64 links); see wilson.cuh.
#include "wilson.cuh"

namespace dgb {
template int launch_wilson_v<double, 1, double>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
}  // namespace dgb
