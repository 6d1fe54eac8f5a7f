// laplace_f32_l1.cu -- one instantiation of the Laplace stencils (f32 vectors and links, layout 1); see laplace.cuh.
#include "laplace.cuh"

namespace dgb {
template int launch_laplace_v<float, 1>(const dirac_op *, const void *, void *, double, cudaStream_t);
}  // namespace dgb
