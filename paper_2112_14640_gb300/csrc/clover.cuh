// clover.cuh -- the site-diagonal end of the D_W and D_B kernels,
//   out(n) = centre psi(n) + coef acc(n)  [+ C(n) psi(n)],
// with the clover term C of Eq. (def_clov), C = -(c_SW/2) sum_{mu<nu} sigma_mu,nu F_mu,nu.
//
// In the chiral basis every sigma_mu,nu is pauli_0 or pauli_3 on the
// chirality index times a Pauli matrix on the two spins of one chirality
// (App. A), so C is block diagonal: for chirality chi (spins 2chi, 2chi+1)
// and e = +1 (chi = 0) or -1 (chi = 1),
//   C_chi = [[ A,    B ],      A = -(c_SW/2) (-F_12 + e F_34),
//            [ B^dag, -A ]],   B = -(c_SW/2) (e F_14 - F_23 - i (F_13 + e F_24)).
// The operator stores A and B per chirality (four N_c x N_c matrices per
// site, c_SW folded in) in the links' layout, matrix index k = 2 chi + (0: A,
// 1: B); applying them costs the two colour multiplications per chiral half
// that App. E counts for the clover term.  C commutes with gamma5, so the
// daggered operator gamma5 (D + C) gamma5 = D^dag + C applies it unchanged.
#pragma once
#include "internal.h"

namespace dgb {

// CLOV = 0: no clover term; 1: clover term; -1: decided at run time by
// clov != nullptr (one uniform branch, for kernels too costly to compile twice).
template <int CLOV, int NC, int VR, int LAYOUT, typename E, typename A, typename EL>
__device__ __forceinline__ void write_site(const E *__restrict__ in, E *__restrict__ out,
                                           const EL *__restrict__ clov, const Lat &g, long long n,
                                           long long base, A centre, A coef, cx<A> (&acc)[NC][4][VR]) {
    using L = Layout<LAYOUT>;
    const long long cs = L::cs_stride(g);
    if (CLOV == 0 || (CLOV < 0 && clov == nullptr)) {
#pragma unroll
        for (int a = 0; a < NC; ++a)
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                cx<A> p[VR], o[VR];
                const long long off = base + 2LL * (a * 4 + s) * cs;
                load_cx<E, VR, A>(in + off, p);
#pragma unroll
                for (int v = 0; v < VR; ++v) {
                    o[v] = centre * p[v];
                    rmac(o[v], coef, acc[a][s][v]);
                }
                store_cx<E, VR, A>(out + off, o);
            }
        return;
    }
    const long long ms = L::template mat_stride<NC>(g);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        // the output of spins 2h, 2h+1 is built in place in acc
        cx<A> p[NC][2][VR];
#pragma unroll
        for (int a = 0; a < NC; ++a)
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                load_cx<E, VR, A>(in + base + 2LL * (a * 4 + 2 * h + t) * cs, p[a][t]);
#pragma unroll
                for (int v = 0; v < VR; ++v) {
                    cx<A> o = centre * p[a][t][v];
                    rmac(o, coef, acc[a][2 * h + t][v]);
                    acc[a][2 * h + t][v] = o;
                }
            }
        cx<A> M[NC][NC];
        // upper-left A, lower-right -A
        load_mat_s<NC, EL, A>(clov + 2 * L::template mat<NC>(g, n, 4, 2 * h), ms, M);
#pragma unroll
        for (int a = 0; a < NC; ++a)
#pragma unroll
            for (int b = 0; b < NC; ++b)
#pragma unroll
                for (int v = 0; v < VR; ++v) {
                    cmac(acc[a][2 * h][v], M[a][b], p[b][0][v]);
                    cmac(acc[a][2 * h + 1][v], cx<A>{-M[a][b].re, -M[a][b].im}, p[b][1][v]);
                }
        // upper-right B, lower-left B^dag
        load_mat_s<NC, EL, A>(clov + 2 * L::template mat<NC>(g, n, 4, 2 * h + 1), ms, M);
#pragma unroll
        for (int a = 0; a < NC; ++a)
#pragma unroll
            for (int b = 0; b < NC; ++b)
#pragma unroll
                for (int v = 0; v < VR; ++v) {
                    cmac(acc[a][2 * h][v], M[a][b], p[b][1][v]);
                    cmac_conj(acc[a][2 * h + 1][v], M[b][a], p[b][0][v]);
                }
#pragma unroll
        for (int a = 0; a < NC; ++a)
#pragma unroll
            for (int t = 0; t < 2; ++t)
                store_cx<E, VR, A>(out + base + 2LL * (a * 4 + 2 * h + t) * cs, acc[a][2 * h + t]);
    }
}

}  // namespace dgb
