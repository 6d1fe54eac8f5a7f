// brillouin.cuh -- multi-RHS Brillouin Dirac operator, Eq. (app_bril) with
// Eqs. (def_ider, def_blap) at r = 1, c_SW = 0:
//   (D_B psi)(n) = (m0 - lambda_0/2) psi(n)
//       + sum_{s in {-1,0,1}^4, s != 0} [sgn rho_k sum_mu s_mu gamma_mu - lambda_k/2] (x) W_s(n) psi(n+s)
// rho = (64,16,4,1)/432, lambda = (-240,8,4,2,1)/64, k = |s|_1, W_s from
// Tab. off-axis, built once per gauge field (links.cu) and stored in the
// order q, with the scale rho_k s_lead and the per-site layout of bril_dirs.h.  The derivative
// carries every axis the offset moves along (sum_mu s_mu gamma_mu), the
// reading of Eq. (def_ider).  sgn = +1 gives D_B, sgn = -1 gives
// D_B^dag = gamma5 D_B gamma5 (the derivative part flips sign).  A clover
// term, when the operator carries one, is added site by site at the end
// (clover.cuh; Eq. def_bril).
//
// With the stored W~ = rho_k s_lead W_s every offset contributes
//   sgn * W~ [ sum_{mu in M} e_mu gamma_mu psi(n+s) + d psi(n+s) ],
//   e_mu = s_lead s_mu,  d = -sgn c_k s_lead,
// and the common factor sgn is applied once to the accumulated sum.  The
// offsets are visited group by group of equal support M (a compile-time
// mask), so the gamma matrices of the axes outside M cost nothing: in the
// chiral basis of App. A each gamma_mu is a signed permutation of the spin
// components, and the spin combination costs 8k real FMAs per colour and RHS
// instead of 40.  Inside a group the 2^k sign patterns run in a loop (two per
// trip), the W~ of the next offset is loaded while the current one is
// applied, and each W~ is used for all 4 spins and the thread's VR
// right-hand sides.
#pragma once
#include "bril_dirs.h"
#include "clover.cuh"
#include "internal.h"

namespace dgb {
namespace bril {

// phase * p[pi] of gamma_mu acting on spin S (chiral basis of App. A):
//   t: pi = (2,3,0,1), phases ( 1,  1, 1,  1)    z: pi = (2,3,0,1), phases (-i, i, i, -i)
//   y: pi = (3,2,1,0), phases (-1,  1, 1, -1)    x: pi = (3,2,1,0), phases (-i, -i, i, i)
template <int MU, int S, typename A>
__device__ __forceinline__ cx<A> gamma_term(const cx<A> (&p)[4]) {
    constexpr int PI = MU >= 2 ? (S ^ 2) : (3 - S);
    // 0: +1, 1: -1, 2: +i, 3: -i
    constexpr int PH = MU == 3 ? 0
                     : MU == 2 ? ((S == 0 || S == 3) ? 3 : 2)
                     : MU == 1 ? ((S == 0 || S == 3) ? 1 : 0)
                               : (S <= 1 ? 3 : 2);
    const cx<A> v = p[PI];
    if constexpr (PH == 0) return v;
    else if constexpr (PH == 1) return cx<A>{-v.re, -v.im};
    else if constexpr (PH == 2) return cx<A>{-v.im, v.re};
    else return cx<A>{v.im, -v.re};
}

// f += e_mu * (gamma_mu p)_S for the axes MU.. of M other than the lead
template <int M, int S, int MU, typename A>
__device__ __forceinline__ void add_axes(cx<A> &f, const cx<A> (&p)[4], const A (&e)[4]) {
    if constexpr (MU < 4) {
        if constexpr (((M >> MU) & 1) && MU != lead_axis(M)) {
            const cx<A> t = gamma_term<MU, S>(p);
            f.re = fma(e[MU], t.re, f.re);
            f.im = fma(e[MU], t.im, f.im);
        }
        add_axes<M, S, MU + 1>(f, p, e);
    }
}

// spin component S of  sum_{mu in M} e_mu gamma_mu p + d p
template <int M, int S, typename A>
__device__ __forceinline__ cx<A> spin_mix(const cx<A> (&p)[4], const A (&e)[4], A d) {
    cx<A> f = gamma_term<lead_axis(M), S>(p);
    add_axes<M, S, 0>(f, p, e);
    f.re = fma(d, p[S].re, f.re);
    f.im = fma(d, p[S].im, f.im);
    return f;
}

// spin component S of  sum_mu e_mu gamma_mu p + d p  for all four axes
// (e_mu = 0 off the support; the run-time-mask path of large N_c)
template <int S, typename A>
__device__ __forceinline__ cx<A> spin_mix_rt(const cx<A> (&p)[4], const A (&e)[4], A d) {
    cx<A> f = {d * p[S].re, d * p[S].im};
    const cx<A> t[4] = {gamma_term<0, S>(p), gamma_term<1, S>(p), gamma_term<2, S>(p), gamma_term<3, S>(p)};
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        f.re = fma(e[mu], t[mu].re, f.re);
        f.im = fma(e[mu], t[mu].im, f.im);
    }
    return f;
}

template <int NC, int VR, typename E, typename EL, int LAYOUT>
struct Ctx {
    using A = typename Acc<E>::T;
    const EL *wp;          // this site's W~ (offset 0, element 0), [q][a][b]
    const E *in;
    int n;                 // output site (volumes are below 2^31 sites)
    long long vbase;       // offset of this thread's RHS inside a site (complex numbers)
    int dp[4], dm[4];      // site-index offsets of n + mu and n - mu (periodic)
    Lat g;
    A sgn;
};

// Offset b (sign pattern) of support M, applied with the W~ in Wcur while the
// next offset's W~ is loaded into Wnext (storage order = visiting order).
template <int M, int NC, int VR, typename E, typename EL, int LAYOUT, typename A>
__device__ __forceinline__ void offset(const Ctx<NC, VR, E, EL, LAYOUT> &C, int q, int b,
                                       const cx<A> (&Wcur)[NC][NC], cx<A> (&Wnext)[NC][NC],
                                       cx<A> (&acc)[NC][4][VR]) {
    using L = Layout<LAYOUT>;
    constexpr int K = popc4(M);
    const A ck = (A)c_lambda(K);
    const long long cs = L::cs_stride(C.g);
    A sig[4] = {1, 1, 1, 1};
    int m = C.n;
    {
        int jbit = 0;
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            if ((M >> mu) & 1) {
                const bool neg = (b >> jbit) & 1;
                sig[mu] = neg ? (A)-1 : (A)1;
                m += neg ? C.dm[mu] : C.dp[mu];
                ++jbit;
            }
        }
    }
    const A sl = sig[lead_axis(M)];
    A e[4];
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) e[mu] = sig[mu] * sl;
    const A d = -C.sgn * ck * sl;

    // one site's W~ are contiguous: compile-time element offsets
    if (q + 1 < 80) load_mat<NC, EL, A>(C.wp + (q + 1) * (2 * NC * NC), Wnext);

    const E *pm = C.in + 2 * (L::vec(C.g, (long long)m, NC * 4, 0) + C.vbase);
#pragma unroll
    for (int kc = 0; kc < NC; ++kc) {
        cx<A> p[4][VR];
#pragma unroll
        for (int s = 0; s < 4; ++s) load_cx<E, VR, A>(pm + 2 * (kc * 4 + s) * cs, p[s]);
#pragma unroll
        for (int v = 0; v < VR; ++v) {
            const cx<A> pv[4] = {p[0][v], p[1][v], p[2][v], p[3][v]};
            const cx<A> f0 = spin_mix<M, 0>(pv, e, d);
            const cx<A> f1 = spin_mix<M, 1>(pv, e, d);
            const cx<A> f2 = spin_mix<M, 2>(pv, e, d);
            const cx<A> f3 = spin_mix<M, 3>(pv, e, d);
#pragma unroll
            for (int a = 0; a < NC; ++a) {
                cmac(acc[a][0][v], Wcur[a][kc], f0);
                cmac(acc[a][1][v], Wcur[a][kc], f1);
                cmac(acc[a][2][v], Wcur[a][kc], f2);
                cmac(acc[a][3][v], Wcur[a][kc], f3);
            }
        }
    }
}

// Large N_c: one offset (support M, sign pattern b, both run-time values) with
// the W~ read one row at a time instead of a register double buffer of N_c^2
// elements; the spin-mixed neighbour spinor of every colour is formed first.
// With e_mu = s_mu s_lead on the axes of M and 0 elsewhere, the spin factor
// is sum_mu e_mu gamma_mu + d (as in `offset`, without compile-time masks).
template <int NC, int VR, typename E, typename EL, int LAYOUT, typename A>
__device__ __forceinline__ void offset_rows(const Ctx<NC, VR, E, EL, LAYOUT> &C, int q, int M, int b,
                                            cx<A> (&acc)[NC][4][VR]) {
    using L = Layout<LAYOUT>;
    const int K = popc4(M);
    const A ck = (A)c_lambda(K);
    const long long cs = L::cs_stride(C.g);
    A sig[4] = {0, 0, 0, 0};
    int m = C.n;
    {
        int jbit = 0;
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            if ((M >> mu) & 1) {
                const bool neg = (b >> jbit) & 1;
                sig[mu] = neg ? (A)-1 : (A)1;
                m += neg ? C.dm[mu] : C.dp[mu];
                ++jbit;
            }
        }
    }
    const A sl = sig[lead_axis(M)];
    A e[4];
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) e[mu] = sig[mu] * sl;
    const A d = -C.sgn * ck * sl;
    const E *pm = C.in + 2 * (L::vec(C.g, (long long)m, NC * 4, 0) + C.vbase);
    cx<A> f[NC][4][VR];
#pragma unroll
    for (int kc = 0; kc < NC; ++kc) {
        cx<A> p[4][VR];
#pragma unroll
        for (int s = 0; s < 4; ++s) load_cx<E, VR, A>(pm + 2 * (kc * 4 + s) * cs, p[s]);
#pragma unroll
        for (int v = 0; v < VR; ++v) {
            const cx<A> pv[4] = {p[0][v], p[1][v], p[2][v], p[3][v]};
            f[kc][0][v] = spin_mix_rt<0>(pv, e, d);
            f[kc][1][v] = spin_mix_rt<1>(pv, e, d);
            f[kc][2][v] = spin_mix_rt<2>(pv, e, d);
            f[kc][3][v] = spin_mix_rt<3>(pv, e, d);
        }
    }
    const EL *wq = C.wp + q * (2 * NC * NC);
#pragma unroll 1
    for (int a = 0; a < NC; ++a) {
        cx<A> wr[NC];
#pragma unroll
        for (int kc = 0; kc < NC; ++kc) wr[kc] = ld1<EL, A>(wq + 2 * (a * NC + kc));
        cx<A> o[4][VR];
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int v = 0; v < VR; ++v) o[s][v] = cx<A>{0, 0};
#pragma unroll
        for (int kc = 0; kc < NC; ++kc)
#pragma unroll
            for (int s = 0; s < 4; ++s)
#pragma unroll
                for (int v = 0; v < VR; ++v) cmac(o[s][v], wr[kc], f[kc][s][v]);
        // run-time row index: add through a compile-time switch over rows
#pragma unroll
        for (int r = 0; r < NC; ++r)
            if (r == a)
#pragma unroll
                for (int s = 0; s < 4; ++s)
#pragma unroll
                    for (int v = 0; v < VR; ++v) acc[r][s][v] = acc[r][s][v] + o[s][v];
    }
}

// The 2^k offsets of support M: their signs run in a loop, everything that
// depends on M alone is fixed at compile time.  Two offsets per trip, so the
// two W~ buffers swap roles without copies (every group has an even count);
// Wc holds the current W~ on entry and on exit.
template <int M, int NC, int VR, typename E, typename EL, int LAYOUT, typename A>
__device__ __forceinline__ void group(const Ctx<NC, VR, E, EL, LAYOUT> &C, int &q, cx<A> (&Wc)[NC][NC],
                                      cx<A> (&acc)[NC][4][VR]) {
    constexpr int K = popc4(M);
    if constexpr (NC > kMaxNcSmall) {
        static_assert(M == 1, "large N_c visits all groups in one run-time loop");
        // every group M = 1..15 and its 2^k sign patterns in run-time loops
#pragma unroll 1
        for (int Mr = 1; Mr <= 15; ++Mr)
#pragma unroll 1
            for (int b = 0; b < (1 << popc4(Mr)); ++b) {
                offset_rows(C, q, Mr, b, acc);
                ++q;
            }
    } else {
        cx<A> Wn[NC][NC];
#pragma unroll 1
        for (int b = 0; b < (1 << K); b += 2) {
            offset<M>(C, q, b, Wc, Wn, acc);
            offset<M>(C, q + 1, b + 1, Wn, Wc, acc);
            q += 2;
        }
    }
}

template <int M, int NC, int VR, typename E, typename EL, int LAYOUT, typename A>
__device__ __forceinline__ void groups_from(const Ctx<NC, VR, E, EL, LAYOUT> &C, int &q, cx<A> (&Wc)[NC][NC],
                                            cx<A> (&acc)[NC][4][VR]) {
    if constexpr (NC > kMaxNcSmall) {
        group<1>(C, q, Wc, acc);   // one run-time loop over all groups
    } else if constexpr (M <= 15) {
        group<M>(C, q, Wc, acc);
        groups_from<M + 1>(C, q, Wc, acc);
    }
}

}  // namespace bril

template <int NC, int VR, typename E, int MINB, int LAYOUT, typename EL>
__global__ void __launch_bounds__(stencil_max_threads(MINB), (MINB > 1 ? 1 : 0))
    brillouin_kernel(const EL *__restrict__ W, const E *__restrict__ in, E *__restrict__ out, Lat g,
                     typename Acc<E>::T centre, typename Acc<E>::T sgn, const EL *__restrict__ clov) {
    using A = typename Acc<E>::T;
    using L = Layout<LAYOUT>;
    const int nchunk = g.nv / VR;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= g.nsites * nchunk) return;
    long long i;
    int j;
    split_tid(tid, nchunk, i, j);
    const long long n = g.n0 + i;
    const Coord c = site_coords(g, n);

    bril::Ctx<NC, VR, E, EL, LAYOUT> C;
    C.g = g;
    C.in = in;
    C.n = (int)n;
    C.sgn = sgn;
    C.vbase = (long long)j * VR;
    // W~ of one site contiguous in visiting order for either vector layout
    C.wp = W + 2LL * n * 80 * NC * NC;
    {
        const int co[4] = {c.x, c.y, c.z, c.t};
        const int ext[4] = {g.nx, g.ny, g.nz, g.nt};
        int stride = 1;
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            C.dp[mu] = (co[mu] == ext[mu] - 1 ? -(ext[mu] - 1) : 1) * stride;
            C.dm[mu] = (co[mu] == 0 ? ext[mu] - 1 : -1) * stride;
            stride *= ext[mu];
        }
    }

    cx<A> acc[NC][4][VR];
#pragma unroll
    for (int a = 0; a < NC; ++a)
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int v = 0; v < VR; ++v) acc[a][s][v] = cx<A>{0, 0};

    cx<A> Wc[NC][NC];
    if constexpr (NC <= kMaxNcSmall) load_mat<NC, EL, A>(C.wp, Wc);
    int q = 0;
    bril::groups_from<1>(C, q, Wc, acc);

    const long long base = 2 * (L::vec(g, n, NC * 4, 0) + (long long)j * VR);
    write_site<-1, NC, VR, LAYOUT, E, A, EL>(in, out, clov, g, n, base, centre, sgn, acc);
}

template <typename E, int LAYOUT, typename EL>
int launch_brillouin_v(const dirac_op *op, const void *in, void *out, double m0, int sgn, cudaStream_t s) {
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
                // m0 - lambda_0 / 2 = m0 + 240/128
                {
                brillouin_kernel<NC, VR, E, MINB, LAYOUT, EL><<<grid_for(threads, block), block, 0, s>>>(
                    (const EL *)op->w, (const E *)in, (E *)out, op->lat, (A)(m0 + 240.0 / 128.0), (A)sgn,
                    (const EL *)op->clover);
                return launch_check("brillouin_kernel");
                }
            }
            });
        });
    });
}

}  // namespace dgb
