// internal.h -- operator handle and launcher prototypes shared by the
// translation units of libdirac.so (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdio.h>

#include <type_traits>
#include <utility>

#include "../../include/dirac.h"
#include "common.cuh"

struct dirac_op {
    dirac_kind kind;
    dirac_geom geom;
    dgb::Lat lat;
    int nc, nv;
    dirac_prec prec;
    long long V;
    long long rows;        // complex rows per RHS column: V*nc*4 (Wilson-type) or V*nc
    size_t vec_bytes;      // bytes of one multi-RHS vector
    size_t link_bytes;     // bytes of the phased link copy
    size_t w_bytes;        // bytes of the 80 W links per site (Brillouin)
    void *links;           // [V][4][nc][nc], boundary phases folded in
    void *w;               // [V][80][nc][nc] (Brillouin only)
    void *clover;          // clover term (clover.cuh), links' shape and layout; null when c_SW = 0
    double csw;            // c_SW folded into `clover`
    void *scratch;         // one vector: intermediate of D^dag D
    void *stage_in;        // host-apply staging buffers (lazy)
    void *stage_out;
    struct dirac_host_pipe *pipe;   // host-apply copy streams and events (lazy)
    double *red_partial;   // reduction partials [red_blocks][nv][2]
    int red_blocks;
    void *solver_ws;       // solver workspace (lazy), solver_ws_bytes long
    size_t solver_ws_bytes;
    void *force_ws;        // Brillouin force: 216 link terms per site (lazy), force_ws_bytes long
    size_t force_ws_bytes;
    dirac_op *inner[4][2]; // lower-precision twins for mixed solves (lazy), by [prec][link storage]
    int vr, minb, block;   // stencil launch variant (RHS per thread, register class, threads per block);
                           // 0 = default
};

namespace dgb {

inline int cuda_check(cudaError_t e, const char *what) {
    if (e != cudaSuccess) {
        fprintf(stderr, "libdirac: %s: %s\n", what, cudaGetErrorString(e));
        cudaGetLastError();   // clear a non-sticky error so it is not blamed on a later call
        return DIRAC_ERR_CUDA;
    }
    return DIRAC_OK;
}
inline int launch_check(const char *what) { return cuda_check(cudaGetLastError(), what); }

inline size_t elem_bytes(dirac_prec p) { return p == DIRAC_F64 ? 8 : p == DIRAC_F32 ? 4 : 2; }

// precision the links and W links are stored in
inline dirac_prec link_prec(const dirac_op *op) {
    return (op->geom.link_storage == DIRAC_LINKS_F32 && (op->prec == DIRAC_BF16 || op->prec == DIRAC_F16))
               ? DIRAC_F32 : op->prec;
}

// dispatch the link element type EL for vectors of element type E
template <typename E, typename F>
int dispatch_link_elem(const dirac_op *op, F &&f) {
    if constexpr (sizeof(E) == 2) {
        if (link_prec(op) == DIRAC_F32) return f((float *)nullptr);
    }
    return f((E *)nullptr);
}

// Largest RHS-vector width (complex numbers per thread) that divides nv and
// gives at most 16-byte loads.
inline int pick_vr(dirac_prec p, int nv) {
    int vr = (int)(16 / (2 * elem_bytes(p)));
    while (vr > 1 && nv % vr) vr /= 2;
    return vr;
}

template <typename F>
int dispatch_prec(dirac_prec p, F &&f) {
    switch (p) {
    case DIRAC_F64: return f((double *)nullptr);
    case DIRAC_F32: return f((float *)nullptr);
    case DIRAC_BF16: return f((__nv_bfloat16 *)nullptr);
    case DIRAC_F16: return f((__half *)nullptr);
    }
    return DIRAC_ERR_UNSUPPORTED_PREC;
}

// Colour counts compiled: 1..8 (the paper's N_c sweep reaches 8 within this
// range).  N_c 5..8 are compiled for FP64 and FP32 storage only (BIG = false
// restricts a dispatch to 1..4, as the 16-bit stencils use it), with one RHS
// per thread and the compiler's own register choice (kMaxNcSmall below).
constexpr int kMaxNc = 8;
constexpr int kMaxNcSmall = 4;
template <bool BIG = true, typename F>
int dispatch_nc(int nc, F &&f) {
    switch (nc) {
    case 1: return f(std::integral_constant<int, 1>{});
    case 2: return f(std::integral_constant<int, 2>{});
    case 3: return f(std::integral_constant<int, 3>{});
    case 4: return f(std::integral_constant<int, 4>{});
    }
    if constexpr (BIG) {
        switch (nc) {
        case 5: return f(std::integral_constant<int, 5>{});
        case 6: return f(std::integral_constant<int, 6>{});
        case 7: return f(std::integral_constant<int, 7>{});
        case 8: return f(std::integral_constant<int, 8>{});
        }
    }
    return DIRAC_ERR_UNSUPPORTED_NC;
}
// N_c compiled for a vector element type (16-bit storage: 1..4)
template <typename E>
constexpr bool big_nc_ok() { return sizeof(E) >= 4; }
inline bool nc_supported(int nc, dirac_prec p) {
    return nc >= 1 && nc <= (p == DIRAC_F64 || p == DIRAC_F32 ? kMaxNc : kMaxNcSmall);
}

// VR values compiled for NC colours: 1, 2, 4 for N_c <= 4; 1 above
template <int NC>
constexpr bool vr_compiled(int vr) { return NC <= kMaxNcSmall || vr == 1; }

template <typename F>
int dispatch_vr(int vr, F &&f) {
    switch (vr) {
    case 1: return f(std::integral_constant<int, 1>{});
    case 2: return f(std::integral_constant<int, 2>{});
    case 4: return f(std::integral_constant<int, 4>{});
    }
    return DIRAC_ERR_INVALID_ARG;
}

// Stencil launch variants: VR right-hand sides per thread and a register
// class MINB: the register cap of MINB resident 128-thread blocks per SM
// (65536 / (128 MINB) registers), compiled as __launch_bounds__(128 MINB, 1)
// so that blocks of up to 128 MINB threads can be launched with it; MINB = 1
// compiles with the plain __launch_bounds__(128) (the compiler's own register
// heuristic, which differs from an explicit minimum of one block).  Every
// (VR, MINB) pair below is compiled for N_c = 3; other N_c have MINB = 1 only.
// Larger blocks cover more consecutive x-rows, so more of the y-neighbours a
// block reads are already in its SM's L1.
constexpr int kStencilBlock = 128;
__host__ __device__ constexpr int stencil_max_threads(int minb) { return minb > 1 ? 128 * minb : 128; }
inline bool variant_compiled(int nc, int vr, int minb) {
    if (vr != 1 && vr != 2 && vr != 4) return false;
    if (nc > kMaxNcSmall) return vr == 1 && minb == 1;
    if (minb == 1) return true;
    return nc == 3 && (minb >= 3 && minb <= 6);
}
inline bool variant_ok(const dirac_op *op, int vr, int minb) {
    return variant_compiled(op->nc, vr, minb) && op->nv % vr == 0;
}

template <typename F>
int dispatch_layout(int layout, F &&f) {
    switch (layout) {
    case DIRAC_LAYOUT_SITE_OUTER: return f(std::integral_constant<int, 0>{});
    case DIRAC_LAYOUT_SITE_INNER: return f(std::integral_constant<int, 1>{});
    }
    return DIRAC_ERR_INVALID_ARG;
}

template <int NC, typename F>
int dispatch_minb(int minb, F &&f) {
    if constexpr (NC != 3) {
        return minb == 1 ? f(std::integral_constant<int, 1>{}) : DIRAC_ERR_INVALID_ARG;
    } else {
        switch (minb) {
        case 1: return f(std::integral_constant<int, 1>{});
        case 3: return f(std::integral_constant<int, 3>{});
        case 4: return f(std::integral_constant<int, 4>{});
        case 5: return f(std::integral_constant<int, 5>{});
        case 6: return f(std::integral_constant<int, 6>{});
        }
        return DIRAC_ERR_INVALID_ARG;
    }
}

// kind properties: the Laplace operators -1/2 Lap + m^2/2 (hermitian), the
// number of spin components per colour of the kind's vectors, and whether the
// kind stencils with the 80 Brillouin W links
inline bool is_laplace(dirac_kind k) { return k >= DIRAC_WLAP && k <= DIRAC_BSUV; }
inline int spins_of(dirac_kind k) { return (k == DIRAC_STAGGERED || k == DIRAC_WSUV || k == DIRAC_BSUV) ? 1 : 4; }
inline bool uses_w(dirac_kind k) { return k == DIRAC_BRILLOUIN || k == DIRAC_BLAP || k == DIRAC_BSUV; }

// (vr, minb, block) an operator launches with: its tuned choice or the default.
inline void launch_variant(const dirac_op *op, int &vr, int &minb, int &block) {
    if (op->vr) {
        vr = op->vr;
        minb = op->minb ? op->minb : 1;
        block = op->block ? op->block : kStencilBlock;
        return;
    }
    // untuned: the widest 16-byte RHS group and, for N_c = 3, the register
    // class and block size the autotuner picks for FP32 on 16^3x32 lattices
    vr = op->nc > kMaxNcSmall ? 1 : pick_vr(op->prec, op->nv);
    minb = 1;
    block = kStencilBlock;
    if (op->nc == 3) {
        if (op->kind == DIRAC_WILSON) {
            minb = vr == 4 ? 3 : 4;
        } else if (op->kind == DIRAC_STAGGERED) {
            minb = 3;
        } else if (op->kind == DIRAC_BRILLOUIN && vr <= 2) {
            minb = 3;
            block = 384;
        }
    }
}

inline unsigned grid_for(long long threads, int block) {
    return (unsigned)((threads + block - 1) / block);
}

// stencils (sgn = +1: D, -1: D^dag)
int launch_wilson(const dirac_op *op, const void *in, void *out, double m0, int sgn, cudaStream_t s);
int launch_staggered(const dirac_op *op, const void *in, void *out, double m0, int sgn, cudaStream_t s);
int launch_brillouin(const dirac_op *op, const void *in, void *out, double m0, int sgn, cudaStream_t s);
// A = -1/2 Lap + m^2/2 for the Laplace kinds (laplace.cuh); m is the mass of A
int launch_laplace(const dirac_op *op, const void *in, void *out, double m, cudaStream_t s);

// link preparation
int launch_phase_links(dirac_op *op, const void *U, dirac_prec u_prec, cudaStream_t s);
int launch_build_w(dirac_op *op, const void *U, dirac_prec u_prec, cudaStream_t s);
// one stout-smearing step of a periodic field [site][mu][a][b] (F64 or F32)
int launch_stout_step(const void *U, void *out, const Lat &g, int nc, dirac_prec prec, double rho, cudaStream_t s);
// chain rule through nsteps stout steps (links.cu): G_V -> G_U, GRAD convention; synchronises s
int launch_stout_backward(const void *U, const void *G_V, void *G_U, const Lat &g, int nc, dirac_prec prec, double rho,
                          int nsteps, cudaStream_t s);
// clover term of c_SW = op->csw from gauge field V into op->clover (allocated)
int launch_build_clover(dirac_op *op, const void *V, dirac_prec v_prec, cudaStream_t s);
// the stored W~ (order and scale of bril_dirs.h) back to W_s in the public order
int launch_unpack_w(const dirac_op *op, void *out, cudaStream_t s);
int launch_convert_links(const dirac_op *src, dirac_op *dst, cudaStream_t s);
// Brillouin fermion force (force_bril.cu): F = P_TA(U K) (mode 0) or G = bc K^dag (mode 1)
int launch_bril_force(dirac_op *op, const void *psi, const void *chi, void *out, int mode, cudaStream_t s);

// BLAS-1 (vectors in precision p with op's shape)
int blas_norm2(const dirac_op *op, dirac_prec p, const void *v, double *out, cudaStream_t s);
int blas_dot(const dirac_op *op, dirac_prec p, const void *u, const void *v, double *out, cudaStream_t s);
// Re <u, v> per column: out[v] (N_v doubles)
int blas_dot_re(const dirac_op *op, dirac_prec p, const void *u, const void *v, double *out, cudaStream_t s);
int blas_norm2_range(const dirac_op *op, dirac_prec p, const void *v, long long site0, long long nsites, double *out,
                     cudaStream_t s);
int blas_dot_range(const dirac_op *op, dirac_prec p, const void *u, const void *v, long long site0, long long nsites,
                   double *out, cudaStream_t s);
int blas_axpy(const dirac_op *op, dirac_prec p, const double *alpha, const void *x, void *y, cudaStream_t s);
// z = a x + b y per RHS; a = as * a_coef[v] (complex pairs) or as when a_coef is null (same for b);
// x or y may be null; z may alias x or y; norm_out (device, nv doubles) receives |z|^2 if non-null.
int blas_axpby(const dirac_op *op, dirac_prec p, void *z, const void *x, const double *a_coef, double as,
               const void *y, const double *b_coef, double bs, double *norm_out, cudaStream_t s);
// x += a p, then p = r + b p (a, b per-RHS complex pairs)
int blas_update_xp(const dirac_op *op, dirac_prec p, void *x, void *pv, const void *r, const double *a,
                   const double *b, cudaStream_t s);
int blas_gamma5(const dirac_op *op, dirac_prec p, void *v, cudaStream_t s);
int blas_fill_hash(const dirac_op *op, dirac_prec p, void *v, unsigned seed, cudaStream_t s);
int blas_convert(const dirac_op *op, const void *src, dirac_prec sp, void *dst, dirac_prec dp, cudaStream_t s);

// operator handle helpers (capi.cu)
int op_apply(const dirac_op *op, const void *in, void *out, double m0, int sgn, cudaStream_t s);
int op_apply_normal(const dirac_op *op, const void *in, void *out, double m0, cudaStream_t s);
// the operator CG iterates with: D^dag D, or A itself for the (hermitian) Laplace kinds
int op_apply_cg(const dirac_op *op, const void *in, void *out, double m0, cudaStream_t s);
int op_alloc(dirac_kind kind, const dirac_geom *g, dirac_op **out);
int op_inner(const dirac_op *op, dirac_prec p, int link_storage, dirac_op **out, cudaStream_t s);
void op_destroy(dirac_op *op);

}  // namespace dgb
