// brillouin_f64_l0.cu -- one instantiation of the brillouin stencil (f64 vectors, layout 0, f64 links); see brillouin.cuh.
#include "brillouin.cuh"

namespace dgb {
template int launch_brillouin_v<double, 0, double>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
}  // namespace dgb
