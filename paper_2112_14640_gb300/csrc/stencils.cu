// stencils.cu -- dispatch of the stencil launchers over storage
// precision, vector layout and link storage.  The kernels live in
// wilson.cuh, staggered.cuh and brillouin.cuh; every combination is
// instantiated in its own small translation unit so the library builds in
// parallel.
#include "internal.h"

namespace dgb {

template <typename E, int LAYOUT, typename EL>
int launch_wilson_v(const dirac_op *op, const void *in, void *out, double m0, int sgn, cudaStream_t s);
template <typename E, int LAYOUT, typename EL>
int launch_staggered_v(const dirac_op *op, const void *in, void *out, double m0, int sgn, cudaStream_t s);
template <typename E, int LAYOUT, typename EL>
int launch_brillouin_v(const dirac_op *op, const void *in, void *out, double m0, int sgn, cudaStream_t s);
template <typename E, int LAYOUT>
int launch_laplace_v(const dirac_op *op, const void *in, void *out, double m, cudaStream_t s);
extern template int launch_laplace_v<double, 0>(const dirac_op *, const void *, void *, double, cudaStream_t);
extern template int launch_laplace_v<double, 1>(const dirac_op *, const void *, void *, double, cudaStream_t);
extern template int launch_laplace_v<float, 0>(const dirac_op *, const void *, void *, double, cudaStream_t);
extern template int launch_laplace_v<float, 1>(const dirac_op *, const void *, void *, double, cudaStream_t);

extern template int launch_wilson_v<double, 0, double>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_wilson_v<double, 1, double>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_wilson_v<float, 0, float>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_wilson_v<float, 1, float>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_wilson_v<__nv_bfloat16, 0, __nv_bfloat16>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_wilson_v<__nv_bfloat16, 0, float>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_wilson_v<__nv_bfloat16, 1, __nv_bfloat16>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_wilson_v<__nv_bfloat16, 1, float>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_wilson_v<__half, 0, __half>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_wilson_v<__half, 0, float>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_wilson_v<__half, 1, __half>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_wilson_v<__half, 1, float>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_staggered_v<double, 0, double>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_staggered_v<double, 1, double>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_staggered_v<float, 0, float>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_staggered_v<float, 1, float>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_staggered_v<__nv_bfloat16, 0, __nv_bfloat16>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_staggered_v<__nv_bfloat16, 0, float>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_staggered_v<__nv_bfloat16, 1, __nv_bfloat16>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_staggered_v<__nv_bfloat16, 1, float>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_staggered_v<__half, 0, __half>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_staggered_v<__half, 0, float>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_staggered_v<__half, 1, __half>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_staggered_v<__half, 1, float>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_brillouin_v<double, 0, double>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_brillouin_v<double, 1, double>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_brillouin_v<float, 0, float>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_brillouin_v<float, 1, float>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_brillouin_v<__nv_bfloat16, 0, __nv_bfloat16>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_brillouin_v<__nv_bfloat16, 0, float>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_brillouin_v<__nv_bfloat16, 1, __nv_bfloat16>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_brillouin_v<__nv_bfloat16, 1, float>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_brillouin_v<__half, 0, __half>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_brillouin_v<__half, 0, float>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_brillouin_v<__half, 1, __half>(const dirac_op *, const void *, void *, double, int, cudaStream_t);
extern template int launch_brillouin_v<__half, 1, float>(const dirac_op *, const void *, void *, double, int, cudaStream_t);

template <template <typename, int, typename> class Tag, typename F>
static int dispatch_all(const dirac_op *op, F &&f) {
    return dispatch_prec(op->prec, [&](auto tag) {
        using E = std::remove_pointer_t<decltype(tag)>;
        return dispatch_layout(op->geom.layout, [&](auto lyc) {
            constexpr int LAYOUT = decltype(lyc)::value;
            return dispatch_link_elem<E>(op, [&](auto ltag) {
                using EL = std::remove_pointer_t<decltype(ltag)>;
                return f(Tag<E, LAYOUT, EL>{});
            });
        });
    });
}

template <typename E, int LAYOUT, typename EL> struct WilsonTag {
    static int run(const dirac_op *op, const void *in, void *out, double m0, int sgn, cudaStream_t s) {
        return launch_wilson_v<E, LAYOUT, EL>(op, in, out, m0, sgn, s);
    }
};
template <typename E, int LAYOUT, typename EL> struct StaggeredTag {
    static int run(const dirac_op *op, const void *in, void *out, double m0, int sgn, cudaStream_t s) {
        return launch_staggered_v<E, LAYOUT, EL>(op, in, out, m0, sgn, s);
    }
};
template <typename E, int LAYOUT, typename EL> struct BrillouinTag {
    static int run(const dirac_op *op, const void *in, void *out, double m0, int sgn, cudaStream_t s) {
        return launch_brillouin_v<E, LAYOUT, EL>(op, in, out, m0, sgn, s);
    }
};

int launch_wilson(const dirac_op *op, const void *in, void *out, double m0, int sgn, cudaStream_t s) {
    return dispatch_all<WilsonTag>(op, [&](auto t) { return decltype(t)::run(op, in, out, m0, sgn, s); });
}

int launch_staggered(const dirac_op *op, const void *in, void *out, double m0, int sgn, cudaStream_t s) {
    return dispatch_all<StaggeredTag>(op, [&](auto t) { return decltype(t)::run(op, in, out, m0, sgn, s); });
}

int launch_brillouin(const dirac_op *op, const void *in, void *out, double m0, int sgn, cudaStream_t s) {
    return dispatch_all<BrillouinTag>(op, [&](auto t) { return decltype(t)::run(op, in, out, m0, sgn, s); });
}

// The Laplace kinds exist in FP64 and FP32 (links in the vector precision).
int launch_laplace(const dirac_op *op, const void *in, void *out, double m, cudaStream_t s) {
    const int lay = op->geom.layout;
    if (op->prec == DIRAC_F64)
        return lay ? launch_laplace_v<double, 1>(op, in, out, m, s) : launch_laplace_v<double, 0>(op, in, out, m, s);
    if (op->prec == DIRAC_F32)
        return lay ? launch_laplace_v<float, 1>(op, in, out, m, s) : launch_laplace_v<float, 0>(op, in, out, m, s);
    return DIRAC_ERR_UNSUPPORTED_PREC;
}

}  // namespace dgb
