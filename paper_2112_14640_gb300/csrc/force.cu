// force.cu -- link derivative of the pseudofermion action
//   S = sum_v Re phi_v^dag (D_W^dag D_W)^-1 phi_v       (the paper has no force; derived)
// Given psi = (D^dag D)^-1 phi and chi = D psi, the two hops of D_W through
// U_mu(n) give, with spin and RHS summed,
//   B_mu(n) = sum psi(n+mu) [(1 - gamma_mu) chi(n)]^dag,
//   C_mu(n) = sum psi(n) [(1 + gamma_mu) chi(n+mu)]^dag,
//   dS = Re sum tr[dU_mu(n) (B_mu(n) + C_mu(n)^dag)].
// mode TA:   F_mu(n) = P_TA(U B - C U^dag), so that dS/deps = Re sum tr[X F] for
//            U -> exp(eps X) U, X in su(Nc);
// mode GRAD: G_mu(n) = bc * (B^dag + C), so that dS = Re sum conj(G) dU for the
//            caller's (unphased) links.
// One thread per (site, mu); the (1 +- gamma_mu) projections use the chiral
// gammas of App. A; everything accumulates in the operator's arithmetic type.
//
// The staggered operator (Eq. def_stag) gives the same final form with
//   B_mu(n) = -eta_mu(n) sum psi(n+mu) chi(n)^dag,  C_mu(n) = eta_mu(n) sum psi(n) chi(n+mu)^dag
// (colour vectors, RHS summed; eta_mu(n+mu) = eta_mu(n) because eta_mu only
// depends on the coordinates before mu).
#include "internal.h"

namespace dgb {

// (1 + a gamma_mu) applied to the 4 spin components p[0..3]
template <typename A>
__device__ __forceinline__ void apply_proj(int mu, A a, const cx<A> p[4], cx<A> q[4]) {
    switch (mu) {
    case 0:   // gamma_1 psi = (-i p3, -i p2, i p1, i p0)
        q[0] = p[0] - a * times_i(p[3]);
        q[1] = p[1] - a * times_i(p[2]);
        q[2] = p[2] + a * times_i(p[1]);
        q[3] = p[3] + a * times_i(p[0]);
        break;
    case 1:   // gamma_2 psi = (-p3, p2, p1, -p0)
        q[0] = p[0] - a * p[3];
        q[1] = p[1] + a * p[2];
        q[2] = p[2] + a * p[1];
        q[3] = p[3] - a * p[0];
        break;
    case 2:   // gamma_3 psi = (-i p2, i p3, i p0, -i p1)
        q[0] = p[0] - a * times_i(p[2]);
        q[1] = p[1] + a * times_i(p[3]);
        q[2] = p[2] + a * times_i(p[0]);
        q[3] = p[3] - a * times_i(p[1]);
        break;
    default:  // gamma_4 psi = (p2, p3, p0, p1)
        q[0] = p[0] + a * p[2];
        q[1] = p[1] + a * p[3];
        q[2] = p[2] + a * p[0];
        q[3] = p[3] + a * p[1];
        break;
    }
}

// F = P_TA(U B - C U^dag) (mode 0) or G = bc (B^dag + C) (mode 1) for link (n, mu)
template <int NC, typename E, int LAYOUT>
__device__ __forceinline__ void force_out(const E *__restrict__ U, E *__restrict__ out, const Lat &g, long long tid,
                                          long long n, int mu, const Coord &c, const cx<typename Acc<E>::T> (&B)[NC][NC],
                                          const cx<typename Acc<E>::T> (&C)[NC][NC], int bc0, int bc1, int bc2, int bc3,
                                          int mode) {
    using L = Layout<LAYOUT>;
    using A = typename Acc<E>::T;
    E *o = out + 2 * (tid * NC * NC);
    if (mode == 1) {   // G = bc (B^dag + C)
        const int coord = mu == 0 ? c.x : mu == 1 ? c.y : mu == 2 ? c.z : c.t;
        const int ext = mu == 0 ? g.nx : mu == 1 ? g.ny : mu == 2 ? g.nz : g.nt;
        const int bcm = mu == 0 ? bc0 : mu == 1 ? bc1 : mu == 2 ? bc2 : bc3;
        const A ph = (coord == ext - 1) ? (A)bcm : (A)1;
        for (int a = 0; a < NC; ++a)
            for (int b = 0; b < NC; ++b) {
                cx<A> gv = conj(B[b][a]) + C[a][b];
                o[2 * (a * NC + b)] = from_acc<E, A>(ph * gv.re);
                o[2 * (a * NC + b) + 1] = from_acc<E, A>(ph * gv.im);
            }
        return;
    }
    // M = U B - C U^dag, U = phased link
    cx<A> Lk[NC][NC], M[NC][NC];
    load_mat_s<NC, E, A>(U + 2 * L::template mat<NC>(g, n, 4, mu), L::template mat_stride<NC>(g), Lk);
    for (int a = 0; a < NC; ++a)
        for (int b = 0; b < NC; ++b) {
            cx<A> acc = {0, 0};
            for (int k = 0; k < NC; ++k) {
                cmac(acc, Lk[a][k], B[k][b]);
                cmac(acc, C[a][k], cx<A>{-Lk[b][k].re, Lk[b][k].im});   // - C U^dag
            }
            M[a][b] = acc;
        }
    // P_TA(M) = (M - M^dag)/2 - tr(M - M^dag)/(2 Nc)
    A trim = 0;
    for (int a = 0; a < NC; ++a) trim += M[a][a].im;
    trim /= (A)NC;
    for (int a = 0; a < NC; ++a)
        for (int b = 0; b < NC; ++b) {
            cx<A> f = {(A)0.5 * (M[a][b].re - M[b][a].re), (A)0.5 * (M[a][b].im + M[b][a].im)};
            if (a == b) f.im -= trim;
            o[2 * (a * NC + b)] = from_acc<E, A>(f.re);
            o[2 * (a * NC + b) + 1] = from_acc<E, A>(f.im);
        }
}

template <int NC, typename E, int LAYOUT>
__global__ void force_kernel(const E *__restrict__ U, const E *__restrict__ psi, const E *__restrict__ chi,
                             E *__restrict__ out, Lat g, int bc0, int bc1, int bc2, int bc3, int mode) {
    using L = Layout<LAYOUT>;
    using A = typename Acc<E>::T;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= g.V * 4) return;
    const long long n = tid / 4;
    const int mu = (int)(tid % 4);
    const Coord c = site_coords(g, n);
    const long long m = neighbour(g, n, c, mu, +1);
    const long long csd = L::cs_stride(g);
    cx<A> B[NC][NC], C[NC][NC];
    for (int a = 0; a < NC; ++a)
        for (int b = 0; b < NC; ++b) B[a][b] = C[a][b] = cx<A>{0, 0};
    for (int v = 0; v < g.nv; ++v) {
        cx<A> pn[NC][4], pm[NC][4], qn[NC][4], qm[NC][4];
        for (int a = 0; a < NC; ++a) {
            cx<A> cn[4], cm[4];
            for (int s = 0; s < 4; ++s) {
                const long long on = 2 * (L::vec(g, n, NC * 4, 0) + (long long)(a * 4 + s) * csd + v);
                const long long om = 2 * (L::vec(g, m, NC * 4, 0) + (long long)(a * 4 + s) * csd + v);
                pn[a][s] = ld1<E, A>(psi + on);
                pm[a][s] = ld1<E, A>(psi + om);
                cn[s] = ld1<E, A>(chi + on);
                cm[s] = ld1<E, A>(chi + om);
            }
            apply_proj<A>(mu, (A)-1, cn, qn[a]);   // (1 - gamma_mu) chi(n)
            apply_proj<A>(mu, (A)1, cm, qm[a]);    // (1 + gamma_mu) chi(n+mu)
        }
        for (int a = 0; a < NC; ++a)
            for (int b = 0; b < NC; ++b)
                for (int s = 0; s < 4; ++s) {
                    cmac(B[a][b], pm[a][s], conj(qn[b][s]));
                    cmac(C[a][b], pn[a][s], conj(qm[b][s]));
                }
    }
    force_out<NC, E, LAYOUT>(U, out, g, tid, n, mu, c, B, C, bc0, bc1, bc2, bc3, mode);
}

template <int NC, typename E, int LAYOUT>
__global__ void force_stag_kernel(const E *__restrict__ U, const E *__restrict__ psi, const E *__restrict__ chi,
                                  E *__restrict__ out, Lat g, int bc0, int bc1, int bc2, int bc3, int mode) {
    using L = Layout<LAYOUT>;
    using A = typename Acc<E>::T;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= g.V * 4) return;
    const long long n = tid / 4;
    const int mu = (int)(tid % 4);
    const Coord c = site_coords(g, n);
    const long long m = neighbour(g, n, c, mu, +1);
    const long long csd = L::cs_stride(g);
    // eta_mu(n) = (-1)^(sum_{nu<mu} (x_nu + 1)), the paper's 1-based convention
    const int e[4] = {0, c.x + 1, c.x + c.y + 2, c.x + c.y + c.z + 3};
    const A eta = (e[mu] & 1) ? (A)-1 : (A)1;
    cx<A> B[NC][NC], C[NC][NC];
    for (int a = 0; a < NC; ++a)
        for (int b = 0; b < NC; ++b) B[a][b] = C[a][b] = cx<A>{0, 0};
    for (int v = 0; v < g.nv; ++v) {
        cx<A> pn[NC], pm[NC], cn[NC], cm[NC];
        for (int a = 0; a < NC; ++a) {
            const long long on = 2 * (L::vec(g, n, NC, 0) + (long long)a * csd + v);
            const long long om = 2 * (L::vec(g, m, NC, 0) + (long long)a * csd + v);
            pn[a] = ld1<E, A>(psi + on);
            pm[a] = ld1<E, A>(psi + om);
            cn[a] = ld1<E, A>(chi + on);
            cm[a] = ld1<E, A>(chi + om);
        }
        for (int a = 0; a < NC; ++a)
            for (int b = 0; b < NC; ++b) {
                cmac(B[a][b], pm[a], conj(cn[b]));
                cmac(C[a][b], pn[a], conj(cm[b]));
            }
    }
    for (int a = 0; a < NC; ++a)
        for (int b = 0; b < NC; ++b) {
            B[a][b] = (-eta) * B[a][b];
            C[a][b] = eta * C[a][b];
        }
    force_out<NC, E, LAYOUT>(U, out, g, tid, n, mu, c, B, C, bc0, bc1, bc2, bc3, mode);
}

}  // namespace dgb

using namespace dgb;

extern "C" int dirac_force(const dirac_op *op, const void *psi, const void *chi, void *force_out, int mode,
                           void *stream) {
    if (!op || !psi || !chi || !force_out) return DIRAC_ERR_INVALID_ARG;
    if ((op->kind != DIRAC_WILSON && op->kind != DIRAC_STAGGERED && op->kind != DIRAC_BRILLOUIN) ||
        (mode != 0 && mode != 1))
        return DIRAC_ERR_INVALID_ARG;
    if (op->clover) return DIRAC_ERR_INVALID_ARG;   // derived without the clover term
    if (((uintptr_t)psi & 15) || ((uintptr_t)chi & 15)) return DIRAC_ERR_ALIGNMENT;
    if (op->prec != DIRAC_F64 && op->prec != DIRAC_F32) return DIRAC_ERR_UNSUPPORTED_PREC;
    cudaStream_t s = (cudaStream_t)stream;
    // the handle owns the Brillouin force's scratch (allocated on first use)
    if (op->kind == DIRAC_BRILLOUIN) return launch_bril_force(const_cast<dirac_op *>(op), psi, chi, force_out, mode, s);
    const bool stag = op->kind == DIRAC_STAGGERED;
    return dispatch_prec(op->prec, [&](auto tag) {
        using E = std::remove_pointer_t<decltype(tag)>;
        if constexpr (sizeof(E) == 2) {
            return (int)DIRAC_ERR_UNSUPPORTED_PREC;
        } else {
            return dispatch_nc(op->nc, [&](auto ncc) {
                constexpr int NC = decltype(ncc)::value;
                return dispatch_layout(op->geom.layout, [&](auto lyc) {
                    constexpr int LAYOUT = decltype(lyc)::value;
                    const long long threads = op->V * 4;
                    const int *bc = op->geom.bc;
                    if (stag)
                        force_stag_kernel<NC, E, LAYOUT><<<grid_for(threads, 128), 128, 0, s>>>(
                            (const E *)op->links, (const E *)psi, (const E *)chi, (E *)force_out, op->lat, bc[0],
                            bc[1], bc[2], bc[3], mode);
                    else
                        force_kernel<NC, E, LAYOUT><<<grid_for(threads, 128), 128, 0, s>>>(
                            (const E *)op->links, (const E *)psi, (const E *)chi, (E *)force_out, op->lat, bc[0],
                            bc[1], bc[2], bc[3], mode);
                    return launch_check(stag ? "force_stag_kernel" : "force_kernel");
                });
            });
        }
    });
}

extern "C" int dirac_force_wilson(const dirac_op *op, const void *psi, const void *chi, void *force_out, int mode,
                                  void *stream) {
    if (op && op->kind != DIRAC_WILSON) return DIRAC_ERR_INVALID_ARG;
    return dirac_force(op, psi, chi, force_out, mode, stream);
}
