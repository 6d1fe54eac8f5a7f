// staggered.cuh -- multi-RHS Susskind (staggered) Dirac operator, Eq. (def_stag):
//   (D_S phi)(n) = m0 phi(n) + 1/2 sum_mu eta_mu(n) [U_mu(n) phi(n+mu) - U_mu(n-mu)^dag phi(n-mu)]
// with eta_1 = 1, eta_2 = (-1)^x, eta_3 = (-1)^(x+y), eta_4 = (-1)^(x+y+z) in
// the paper's 1-based coordinates (App. D starts the toggles at x = 1, which
// makes eta_2 = -1 there); with the 0-based coordinates used here the
// exponent is sum_{nu<mu} (x_nu + 1).  D_S^dag = epsilon D_S epsilon flips the
// sign of the anti-hermitian hopping term (sgn = -1).
//
// Thread <-> (site, VR consecutive right-hand sides), colour-vector
// accumulator in registers, one write per output element.
#pragma once
#include "internal.h"

namespace dgb {

template <int NC, int VR, bool DAG, typename E, typename A>
__device__ __forceinline__ void stag_hop_m(cx<A> (&acc)[NC][VR], const cx<A> (&L)[NC][NC],
                                           const E *__restrict__ phi, long long cs_stride, A f);

template <int NC, int VR, bool DAG, typename E, typename A, typename EL>
__device__ __forceinline__ void stag_hop(cx<A> (&acc)[NC][VR], const EL *__restrict__ link, long long lstride,
                                         const E *__restrict__ phi, long long cs_stride, A f) {
    if constexpr (NC > kMaxNcSmall) {
        // large N_c: the link is read one row (column for the dagger) at a time
        cx<A> p[NC][VR];
#pragma unroll
        for (int c = 0; c < NC; ++c) load_cx<E, VR, A>(phi + 2 * c * cs_stride, p[c]);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            cx<A> Lr[NC];
#pragma unroll
            for (int k = 0; k < NC; ++k) Lr[k] = ld1<EL, A>(link + 2 * lstride * (DAG ? k * NC + c : c * NC + k));
#pragma unroll
            for (int v = 0; v < VR; ++v) {
                cx<A> t = {0, 0};
#pragma unroll
                for (int k = 0; k < NC; ++k) {
                    if constexpr (DAG) cmac_conj(t, Lr[k], p[k][v]);
                    else cmac(t, Lr[k], p[k][v]);
                }
                rmac(acc[c][v], f, t);
            }
        }
        return;
    }
    cx<A> L[NC][NC];
    load_mat_s<NC, EL, A>(link, lstride, L);
    stag_hop_m<NC, VR, DAG, E, A>(acc, L, phi, cs_stride, f);
}

// One hop with the link matrix already in registers (N_c <= 4).
template <int NC, int VR, bool DAG, typename E, typename A>
__device__ __forceinline__ void stag_hop_m(cx<A> (&acc)[NC][VR], const cx<A> (&L)[NC][NC],
                                           const E *__restrict__ phi, long long cs_stride, A f) {
    cx<A> p[NC][VR];
#pragma unroll
    for (int c = 0; c < NC; ++c) load_cx<E, VR, A>(phi + 2 * c * cs_stride, p[c]);
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int v = 0; v < VR; ++v) {
            cx<A> t = {0, 0};
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                if constexpr (DAG) cmac_conj(t, L[k][c], p[k][v]);
                else cmac(t, L[c][k], p[k][v]);
            }
            rmac(acc[c][v], f, t);
        }
}

template <int NC, int VR, typename E, int MINB, int LAYOUT, typename EL>
__global__ void __launch_bounds__(stencil_max_threads(MINB), (MINB > 1 ? 1 : 0)) staggered_kernel(const EL *__restrict__ U, const E *__restrict__ in,
                                                        E *__restrict__ out, Lat g, typename Acc<E>::T mass,
                                                        typename Acc<E>::T half_sgn) {
    using A = typename Acc<E>::T;
    const int nchunk = g.nv / VR;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= g.nsites * nchunk) return;
    long long i;
    int j;
    split_tid(tid, nchunk, i, j);
    const long long n = g.n0 + i;
    const Coord c = site_coords(g, n);
    using L = Layout<LAYOUT>;
    const long long cs = L::cs_stride(g), ls = L::template mat_stride<NC>(g);

    cx<A> acc[NC][VR];
#pragma unroll
    for (int a = 0; a < NC; ++a)
#pragma unroll
        for (int v = 0; v < VR; ++v) acc[a][v] = cx<A>{0, 0};

    // eta exponents sum_{nu<mu} (x_nu + 1)
    const int e[4] = {0, c.x + 1, c.x + c.y + 2, c.x + c.y + c.z + 3};
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        const A eta = (e[mu] & 1) ? (A)-1 : (A)1;
        const long long fw = neighbour(g, n, c, mu, +1);
        const long long bw = neighbour(g, n, c, mu, -1);
        if constexpr (NC <= kMaxNcSmall) {
            // both links of the direction requested before either hop
            cx<A> Lf[NC][NC], Lb[NC][NC];
            load_mat_s<NC, EL, A>(U + 2 * L::template mat<NC>(g, n, 4, mu), ls, Lf);
            load_mat_s<NC, EL, A>(U + 2 * L::template mat<NC>(g, bw, 4, mu), ls, Lb);
            stag_hop_m<NC, VR, false, E, A>(acc, Lf, in + 2 * (L::vec(g, fw, NC, 0) + (long long)j * VR), cs, eta);
            stag_hop_m<NC, VR, true, E, A>(acc, Lb, in + 2 * (L::vec(g, bw, NC, 0) + (long long)j * VR), cs, -eta);
        } else {
            stag_hop<NC, VR, false>(acc, U + 2 * L::template mat<NC>(g, n, 4, mu), ls,
                                    in + 2 * (L::vec(g, fw, NC, 0) + (long long)j * VR), cs, eta);
            stag_hop<NC, VR, true>(acc, U + 2 * L::template mat<NC>(g, bw, 4, mu), ls,
                                   in + 2 * (L::vec(g, bw, NC, 0) + (long long)j * VR), cs, -eta);
        }
    }

    const long long base = 2 * (L::vec(g, n, NC, 0) + (long long)j * VR);
#pragma unroll
    for (int a = 0; a < NC; ++a) {
        cx<A> p[VR], o[VR];
        const long long off = base + 2LL * a * cs;
        load_cx<E, VR, A>(in + off, p);
#pragma unroll
        for (int v = 0; v < VR; ++v) {
            o[v] = mass * p[v];
            rmac(o[v], half_sgn, acc[a][v]);
        }
        store_cx<E, VR, A>(out + off, o);
    }
}

template <typename E, int LAYOUT, typename EL>
int launch_staggered_v(const dirac_op *op, const void *in, void *out, double m0, int sgn, cudaStream_t s) {
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
            {
                const long long threads = op->lat.nsites * (op->nv / VR);
                {
                staggered_kernel<NC, VR, E, MINB, LAYOUT, EL><<<grid_for(threads, block), block, 0, s>>>(
                    (const EL *)op->links, (const E *)in, (E *)out, op->lat, (A)m0, (A)(0.5 * sgn));
                return launch_check("staggered_kernel");
                }
            }
            });
        });
    });
}

}  // namespace dgb
