// laplace_f64_l0.cu -- one instantiation of the Laplace stencils (f64 vectors and links, layout 0); see laplace.cuh.
#include "laplace.cuh"

namespace dgb {
template int launch_laplace_v<double, 0>(const dirac_op *, const void *, void *, double, cudaStream_t);
}  // namespace dgb
