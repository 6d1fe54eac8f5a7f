// stencils.cu -- precision dispatch of the three stencil launchers; the
// kernels live in wilson.cuh, staggered.cuh and brillouin.cuh and are
// instantiated one precision per translation unit so they compile in parallel.
#include "internal.h"

namespace dgb {

template <typename E>
int launch_wilson_t(const dirac_op *op, const void *in, void *out, double m0, int sgn, cudaStream_t s);
template <typename E>
int launch_staggered_t(const dirac_op *op, const void *in, void *out, double m0, int sgn, cudaStream_t s);
template <typename E>
int launch_brillouin_t(const dirac_op *op, const void *in, void *out, double m0, int sgn, cudaStream_t s);

extern template int launch_wilson_t<double>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_wilson_t<float>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_wilson_t<__nv_bfloat16>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_wilson_t<__half>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_staggered_t<double>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_staggered_t<float>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_staggered_t<__nv_bfloat16>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_staggered_t<__half>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_brillouin_t<double>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_brillouin_t<float>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_brillouin_t<__nv_bfloat16>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_brillouin_t<__half>(const dirac_op *, const void *, void *, double, int, cudaStream_t);

int launch_wilson(const dirac_op *op, const void *in, void *out, double m0, int sgn, cudaStream_t s) {
    return dispatch_prec(op->prec, [&](auto tag) {
        using E = std::remove_pointer_t<decltype(tag)>;
        return launch_wilson_t<E>(op, in, out, m0, sgn, s);
    });
}

int launch_staggered(const dirac_op *op, const void *in, void *out, double m0, int sgn, cudaStream_t s) {
    return dispatch_prec(op->prec, [&](auto tag) {
        using E = std::remove_pointer_t<decltype(tag)>;
        return launch_staggered_t<E>(op, in, out, m0, sgn, s);
    });
}

int launch_brillouin(const dirac_op *op, const void *in, void *out, double m0, int sgn, cudaStream_t s) {
    return dispatch_prec(op->prec, [&](auto tag) {
        using E = std::remove_pointer_t<decltype(tag)>;
        return launch_brillouin_t<E>(op, in, out, m0, sgn, s);
    });
}

}  // namespace dgb
