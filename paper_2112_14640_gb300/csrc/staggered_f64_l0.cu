// staggered_f64_l0.cu -- one instantiation of the staggered stencil (f64 vectors, layout 0, f64 links); see staggered.cuh.
#include "staggered.cuh"

namespace dgb {
template int launch_staggered_v<double, 0, double>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
}  // namespace dgb
