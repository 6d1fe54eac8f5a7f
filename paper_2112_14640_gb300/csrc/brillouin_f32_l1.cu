// brillouin_f32_l1.cu -- one instantiation of the brillouin stencil (f32 vectors, layout 1, f32 links); see brillouin.cuh.
#include "brillouin.cuh"

namespace dgb {
template int launch_brillouin_v<float, 1, float>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
}  // namespace dgb
