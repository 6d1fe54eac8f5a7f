// wilson.cuh -- multi-RHS Wilson Dirac operator, Eq. (app_wils) at r = 1,
// c_SW = 0:
//   (D_W psi)(n) = (4 + m0) psi(n)
//       - 1/2 sum_mu { (1 - gamma_mu) U_mu(n) psi(n+mu) + (1 + gamma_mu) U_mu(n-mu)^dag psi(n-mu) }
// with the spin-projection trick of App. A: each projector (1 +- gamma_mu)
// has rank two, so the colour multiplication acts on a two-component half
// spinor h and the lower two spin components are rebuilt from h.  The dagger
// D_W^dag = gamma5 D_W gamma5 only swaps the two projectors (sgn = -1).
//
// Thread <-> (output site n, group of VR consecutive right-hand sides): the
// RHS index is innermost in memory, so the VR complex numbers of one
// (colour, spin) component are one 16-byte load and neighbouring threads read
// neighbouring bytes.  Every thread accumulates its whole output in
// registers and writes it once (the paper's write-once "site" accumulator).
#pragma once
#include "clover.cuh"
#include "internal.h"

namespace dgb {

// (1 + a gamma_mu) psi = [h0, h1, r2(h), r3(h)] in the chiral basis; returns
// the half spinor h from the four spin components of one colour.
template <int MU, typename A>
__device__ __forceinline__ void project(const cx<A> p0, const cx<A> p1, const cx<A> p2, const cx<A> p3, A a,
                                        cx<A> &h0, cx<A> &h1) {
    if constexpr (MU == 0) {          // gamma_1 psi = (-i p3, -i p2, i p1, i p0)
        h0 = p0 - a * times_i(p3);
        h1 = p1 - a * times_i(p2);
    } else if constexpr (MU == 1) {   // gamma_2 psi = (-p3, p2, p1, -p0)
        h0 = p0 - a * p3;
        h1 = p1 + a * p2;
    } else if constexpr (MU == 2) {   // gamma_3 psi = (-i p2, i p3, i p0, -i p1)
        h0 = p0 - a * times_i(p2);
        h1 = p1 + a * times_i(p3);
    } else {                          // gamma_4 psi = (p2, p3, p0, p1)
        h0 = p0 + a * p2;
        h1 = p1 + a * p3;
    }
}

// acc += (1 + a gamma_mu) expanded from the colour-multiplied half spinor.
template <int MU, typename A>
__device__ __forceinline__ void reconstruct(cx<A> &o0, cx<A> &o1, cx<A> &o2, cx<A> &o3, const cx<A> c0,
                                            const cx<A> c1, A a) {
    o0 = o0 + c0;
    o1 = o1 + c1;
    if constexpr (MU == 0) {
        o2 = o2 + a * times_i(c1);
        o3 = o3 + a * times_i(c0);
    } else if constexpr (MU == 1) {
        o2 = o2 + a * c1;
        o3 = o3 - a * c0;
    } else if constexpr (MU == 2) {
        o2 = o2 + a * times_i(c0);
        o3 = o3 - a * times_i(c1);
    } else {
        o2 = o2 + a * c0;
        o3 = o3 + a * c1;
    }
}

template <int MU, bool DAG, int NC, int VR, typename E, typename A>
__device__ __forceinline__ void wilson_hop_m(cx<A> (&acc)[NC][4][VR], const cx<A> (&L)[NC][NC],
                                             const E *__restrict__ psi, long long cs_stride, A a);

// One hop: acc += (1 + a gamma_MU) (x) L psi(m), L = link or link^dag.  The
// link elements are lstride complex numbers apart, the spinor components
// cs_stride apart (both depend on the layout).
template <int MU, bool DAG, int NC, int VR, typename E, typename A, typename EL>
__device__ __forceinline__ void wilson_hop(cx<A> (&acc)[NC][4][VR], const EL *__restrict__ link, long long lstride,
                                           const E *__restrict__ psi, long long cs_stride, A a) {
    if constexpr (NC > kMaxNcSmall) {
        // large N_c: project first, then read the link one row (column for
        // the dagger) at a time instead of holding all N_c^2 elements
        cx<A> h[NC][2][VR];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            cx<A> p[4][VR];
#pragma unroll
            for (int s = 0; s < 4; ++s) load_cx<E, VR, A>(psi + 2 * (c * 4 + s) * cs_stride, p[s]);
#pragma unroll
            for (int v = 0; v < VR; ++v) project<MU, A>(p[0][v], p[1][v], p[2][v], p[3][v], a, h[c][0][v], h[c][1][v]);
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            cx<A> Lr[NC];
#pragma unroll
            for (int k = 0; k < NC; ++k) Lr[k] = ld1<EL, A>(link + 2 * lstride * (DAG ? k * NC + c : c * NC + k));
#pragma unroll
            for (int v = 0; v < VR; ++v) {
                cx<A> c0 = {0, 0}, c1 = {0, 0};
#pragma unroll
                for (int k = 0; k < NC; ++k) {
                    if constexpr (DAG) {
                        cmac_conj(c0, Lr[k], h[k][0][v]);
                        cmac_conj(c1, Lr[k], h[k][1][v]);
                    } else {
                        cmac(c0, Lr[k], h[k][0][v]);
                        cmac(c1, Lr[k], h[k][1][v]);
                    }
                }
                reconstruct<MU, A>(acc[c][0][v], acc[c][1][v], acc[c][2][v], acc[c][3][v], c0, c1, a);
            }
        }
        return;
    }
    cx<A> L[NC][NC];
    load_mat_s<NC, EL, A>(link, lstride, L);
    wilson_hop_m<MU, DAG, NC, VR, E, A>(acc, L, psi, cs_stride, a);
}

// One hop with the link matrix already in registers (N_c <= 4).
template <int MU, bool DAG, int NC, int VR, typename E, typename A>
__device__ __forceinline__ void wilson_hop_m(cx<A> (&acc)[NC][4][VR], const cx<A> (&L)[NC][NC],
                                             const E *__restrict__ psi, long long cs_stride, A a) {
    cx<A> h[NC][2][VR];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        cx<A> p[4][VR];
#pragma unroll
        for (int s = 0; s < 4; ++s) load_cx<E, VR, A>(psi + 2 * (c * 4 + s) * cs_stride, p[s]);
#pragma unroll
        for (int v = 0; v < VR; ++v) project<MU, A>(p[0][v], p[1][v], p[2][v], p[3][v], a, h[c][0][v], h[c][1][v]);
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
#pragma unroll
        for (int v = 0; v < VR; ++v) {
            cx<A> c0 = {0, 0}, c1 = {0, 0};
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                if constexpr (DAG) {
                    cmac_conj(c0, L[k][c], h[k][0][v]);
                    cmac_conj(c1, L[k][c], h[k][1][v]);
                } else {
                    cmac(c0, L[c][k], h[k][0][v]);
                    cmac(c1, L[c][k], h[k][1][v]);
                }
            }
            reconstruct<MU, A>(acc[c][0][v], acc[c][1][v], acc[c][2][v], acc[c][3][v], c0, c1, a);
        }
    }
}

template <int MU, int NC, int VR, int LAYOUT, typename E, typename A, typename EL>
__device__ __forceinline__ void wilson_dir(cx<A> (&acc)[NC][4][VR], const EL *__restrict__ U,
                                           const E *__restrict__ in, const Lat &g, long long n, const Coord &c,
                                           int j, A sgn) {
    using L = Layout<LAYOUT>;
    const long long fw = neighbour(g, n, c, MU, +1);
    const long long bw = neighbour(g, n, c, MU, -1);
    const long long cs = L::cs_stride(g), ls = L::template mat_stride<NC>(g);
    if constexpr (NC <= kMaxNcSmall) {
        // both links of the direction are requested before either hop, so
        // their loads are in flight together
        cx<A> Lf[NC][NC], Lb[NC][NC];
        load_mat_s<NC, EL, A>(U + 2 * L::template mat<NC>(g, n, 4, MU), ls, Lf);
        load_mat_s<NC, EL, A>(U + 2 * L::template mat<NC>(g, bw, 4, MU), ls, Lb);
        // forward: (1 - sgn gamma) U_mu(n) psi(n+mu); backward: (1 + sgn gamma) U_mu(n-mu)^dag psi(n-mu)
        wilson_hop_m<MU, false, NC, VR, E, A>(acc, Lf, in + 2 * (L::vec(g, fw, NC * 4, 0) + (long long)j * VR), cs,
                                              -sgn);
        wilson_hop_m<MU, true, NC, VR, E, A>(acc, Lb, in + 2 * (L::vec(g, bw, NC * 4, 0) + (long long)j * VR), cs,
                                             sgn);
    } else {
        wilson_hop<MU, false, NC, VR>(acc, U + 2 * L::template mat<NC>(g, n, 4, MU), ls,
                                      in + 2 * (L::vec(g, fw, NC * 4, 0) + (long long)j * VR), cs, -sgn);
        wilson_hop<MU, true, NC, VR>(acc, U + 2 * L::template mat<NC>(g, bw, 4, MU), ls,
                                     in + 2 * (L::vec(g, bw, NC * 4, 0) + (long long)j * VR), cs, sgn);
    }
}

template <int NC, int VR, typename E, int MINB, int LAYOUT, typename EL, int CLOV>
__global__ void __launch_bounds__(stencil_max_threads(MINB), (MINB > 1 ? 1 : 0)) wilson_kernel(const EL *__restrict__ U, const E *__restrict__ in,
                                                     E *__restrict__ out, Lat g, typename Acc<E>::T diag,
                                                     typename Acc<E>::T sgn, const EL *__restrict__ clov) {
    using A = typename Acc<E>::T;
    const int nchunk = g.nv / VR;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= g.nsites * nchunk) return;
    long long i;
    int j;
    split_tid(tid, nchunk, i, j);
    const long long n = g.n0 + i;
    const Coord c = site_coords(g, n);

    cx<A> acc[NC][4][VR];
#pragma unroll
    for (int a = 0; a < NC; ++a)
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int v = 0; v < VR; ++v) acc[a][s][v] = cx<A>{0, 0};

    wilson_dir<0, NC, VR, LAYOUT, E, A, EL>(acc, U, in, g, n, c, j, sgn);
    wilson_dir<1, NC, VR, LAYOUT, E, A, EL>(acc, U, in, g, n, c, j, sgn);
    wilson_dir<2, NC, VR, LAYOUT, E, A, EL>(acc, U, in, g, n, c, j, sgn);
    wilson_dir<3, NC, VR, LAYOUT, E, A, EL>(acc, U, in, g, n, c, j, sgn);

    const long long base = 2 * (Layout<LAYOUT>::vec(g, n, NC * 4, 0) + (long long)j * VR);
    write_site<CLOV, NC, VR, LAYOUT, E, A, EL>(in, out, clov, g, n, base, diag, (A)-0.5, acc);
}

template <typename E, int LAYOUT, typename EL>
int launch_wilson_v(const dirac_op *op, const void *in, void *out, double m0, int sgn, cudaStream_t s) {
    int vr, minb, block;
    launch_variant(op, vr, minb, block);
    using A = typename Acc<E>::T;
    return dispatch_nc<big_nc_ok<E>()>(op->nc, [&](auto ncc) {
        constexpr int NC = decltype(ncc)::value;
        return dispatch_vr(vr, [&](auto vrc) {
            constexpr int VR = decltype(vrc)::value;
            if constexpr (!vr_compiled<NC>(VR)) return (int)DIRAC_ERR_INVALID_ARG;
            else return dispatch_minb<NC>(minb, [&](auto mbc) {
                constexpr int MINB = decltype(mbc)::value;
                const long long threads = op->lat.nsites * (op->nv / VR);
                // the clover term is a compile-time switch here (no cost to D_W without it)
                auto go = [&](auto cl) {
                    wilson_kernel<NC, VR, E, MINB, LAYOUT, EL, decltype(cl)::value>
                        <<<grid_for(threads, block), block, 0, s>>>((const EL *)op->links, (const E *)in, (E *)out,
                                                                   op->lat, (A)(4.0 + m0), (A)sgn,
                                                                   (const EL *)op->clover);
                    return launch_check("wilson_kernel");
                };
                return op->clover ? go(std::integral_constant<int, 1>{}) : go(std::integral_constant<int, 0>{});
            });
        });
    });
}

}  // namespace dgb
