// brillouin.cuh -- multi-RHS Brillouin Dirac operator, Eq. (app_bril) with
// Eqs. (def_ider, def_blap) at r = 1, c_SW = 0:
//   (D_B psi)(n) = (m0 - lambda_0/2) psi(n)
//       + sum_{s in {-1,0,1}^4, s != 0} [rho_k sum_mu s_mu gamma_mu - lambda_k/2] (x) W_s(n) psi(n+s)
// rho = (64,16,4,1)/432, lambda = (-240,8,4,2,1)/64, k = |s|_1, W_s from
// Tab. off-axis (built once per gauge field in links.cu, all 80 directions
// stored so every output site streams its own W links).  The derivative
// carries every axis the offset moves along (sum_mu s_mu gamma_mu), the
// reading of Eq. (def_ider).  D_B^dag = gamma5 D_B gamma5 flips the sign of
// the derivative part only (sgn = -1).
//
// Per offset the spin matrix Gamma_s = G - l with G = sum_mu a_mu gamma_mu
// acts first, in the chiral basis of App. A:
//   G psi = ( conj(P) p2 - Q p3,  conj(Q) p2 + P p3,  P p0 + Q p1,  -conj(Q) p0 + conj(P) p1 ),
//   P = a_t + i a_z,  Q = a_y + i a_x,
// then the colour matrix W_s(n) multiplies the result into the register
// accumulator; each W_s(n) is loaded once and used for all 4 spins and the
// thread's VR right-hand sides.
#pragma once
#include "internal.h"

namespace dgb {

template <int NC, int VR, typename E, int MINB, int LAYOUT, typename EL>
__global__ void __launch_bounds__(stencil_max_threads(MINB), (MINB > 1 ? 1 : 0)) brillouin_kernel(const EL *__restrict__ W, const E *__restrict__ in,
                                                        E *__restrict__ out, Lat g, typename Acc<E>::T centre,
                                                        typename Acc<E>::T sgn) {
    using A = typename Acc<E>::T;
    const int nchunk = g.nv / VR;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= g.V * nchunk) return;
    const long long n = tid / nchunk;
    const int j = (int)(tid - n * nchunk);
    const Coord c = site_coords(g, n);
    using L = Layout<LAYOUT>;
    const long long cs = L::cs_stride(g), ws = L::mat_stride(g);

    cx<A> acc[NC][4][VR];
#pragma unroll
    for (int a = 0; a < NC; ++a)
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int v = 0; v < VR; ++v) acc[a][s][v] = cx<A>{0, 0};

    const int xs[3] = {c.x == 0 ? g.nx - 1 : c.x - 1, c.x, c.x == g.nx - 1 ? 0 : c.x + 1};
    const int ys[3] = {c.y == 0 ? g.ny - 1 : c.y - 1, c.y, c.y == g.ny - 1 ? 0 : c.y + 1};
    const int zs[3] = {c.z == 0 ? g.nz - 1 : c.z - 1, c.z, c.z == g.nz - 1 ? 0 : c.z + 1};
    const int ts[3] = {c.t == 0 ? g.nt - 1 : c.t - 1, c.t, c.t == g.nt - 1 ? 0 : c.t + 1};

    for (int it = 0; it < 3; ++it) {
        for (int iz = 0; iz < 3; ++iz) {
            const long long tz = (long long)ts[it] * g.nz + zs[iz];
            for (int iy = 0; iy < 3; ++iy) {
                const long long tzy = tz * g.ny + ys[iy];
#pragma unroll
                for (int ix = 0; ix < 3; ++ix) {
                    const int dir = it * 27 + iz * 9 + iy * 3 + ix;
                    if (dir == 40) continue;
                    const int dirp = dir < 40 ? dir : dir - 1;
                    const int k = (it != 1) + (iz != 1) + (iy != 1) + (ix != 1);
                    const A rho = k == 1 ? (A)(64.0 / 432.0) : k == 2 ? (A)(16.0 / 432.0)
                                : k == 3 ? (A)(4.0 / 432.0) : (A)(1.0 / 432.0);
                    const A l = k == 1 ? (A)(8.0 / 128.0) : k == 2 ? (A)(4.0 / 128.0)
                              : k == 3 ? (A)(2.0 / 128.0) : (A)(1.0 / 128.0);
                    const A sr = sgn * rho;
                    const cx<A> P = {sr * (A)(it - 1), sr * (A)(iz - 1)};
                    const cx<A> Q = {sr * (A)(iy - 1), sr * (A)(ix - 1)};
                    const cx<A> mQ = {-Q.re, -Q.im};
                    const A ml = -l;

                    cx<A> Wm[NC][NC];
                    load_mat_s<NC, EL, A>(W + 2 * L::template mat<NC>(g, n, 80, dirp), ws, Wm);
                    const long long m = tzy * g.nx + xs[ix];
                    const E *pm = in + 2 * (L::vec(g, m, NC * 4, 0) + (long long)j * VR);
#pragma unroll
                    for (int kc = 0; kc < NC; ++kc) {
                        cx<A> p[4][VR];
#pragma unroll
                        for (int s = 0; s < 4; ++s) load_cx<E, VR, A>(pm + 2 * (kc * 4 + s) * cs, p[s]);
#pragma unroll
                        for (int v = 0; v < VR; ++v) {
                            cx<A> f0 = ml * p[0][v], f1 = ml * p[1][v], f2 = ml * p[2][v], f3 = ml * p[3][v];
                            cmac_conj(f0, P, p[2][v]);
                            cmac(f0, mQ, p[3][v]);
                            cmac_conj(f1, Q, p[2][v]);
                            cmac(f1, P, p[3][v]);
                            cmac(f2, P, p[0][v]);
                            cmac(f2, Q, p[1][v]);
                            cmac_conj(f3, mQ, p[0][v]);
                            cmac_conj(f3, P, p[1][v]);
#pragma unroll
                            for (int a = 0; a < NC; ++a) {
                                cmac(acc[a][0][v], Wm[a][kc], f0);
                                cmac(acc[a][1][v], Wm[a][kc], f1);
                                cmac(acc[a][2][v], Wm[a][kc], f2);
                                cmac(acc[a][3][v], Wm[a][kc], f3);
                            }
                        }
                    }
                }
            }
        }
    }

    const long long base = 2 * (L::vec(g, n, NC * 4, 0) + (long long)j * VR);
#pragma unroll
    for (int a = 0; a < NC; ++a)
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            cx<A> p[VR], o[VR];
            const long long off = base + 2LL * (a * 4 + s) * cs;
            load_cx<E, VR, A>(in + off, p);
#pragma unroll
            for (int v = 0; v < VR; ++v) {
                o[v] = acc[a][s][v];
                rmac(o[v], centre, p[v]);
            }
            store_cx<E, VR, A>(out + off, o);
        }
}

template <typename E, int LAYOUT, typename EL>
int launch_brillouin_v(const dirac_op *op, const void *in, void *out, double m0, int sgn, cudaStream_t s) {
    int vr, minb, block;
    launch_variant(op, vr, minb, block);
    using A = typename Acc<E>::T;
    return dispatch_nc(op->nc, [&](auto ncc) {
        constexpr int NC = decltype(ncc)::value;
        return dispatch_vr(vr, [&](auto vrc) {
            constexpr int VR = decltype(vrc)::value;
            return dispatch_minb<NC>(minb, [&](auto mbc) {
            constexpr int MINB = decltype(mbc)::value;
            {
                const long long threads = op->V * (op->nv / VR);
                // m0 - lambda_0 / 2 = m0 + 240/128
                {
                brillouin_kernel<NC, VR, E, MINB, LAYOUT, EL><<<grid_for(threads, block), block, 0, s>>>(
                    (const EL *)op->w, (const E *)in, (E *)out, op->lat, (A)(m0 + 240.0 / 128.0), (A)sgn);
                return launch_check("brillouin_kernel");
                }
            }
            });
        });
    });
}

}  // namespace dgb
