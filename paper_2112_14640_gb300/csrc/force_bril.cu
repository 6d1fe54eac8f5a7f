// force_bril.cu -- link derivative of the pseudofermion action for the
// Brillouin operator (the paper has no force; derived here):
//   S = sum_v Re phi_v^dag (D_B^dag D_B)^-1 phi_v,  psi = (D^dag D)^-1 phi,  chi = D_B psi.
// From Eq. (app_bril), dS = -2 Re <chi, dD psi> and
//   dD psi(n) = sum_s S_s (x) dW_s(n) psi(n+s),  S_s = rho_k sum_mu s_mu gamma_mu - lambda_k/2,
// so dS = Re sum_{n,s} tr[dW_s(n) G_s(n)] with G_s = -2 M_s,
//   M_s(n) = sum_{v, spin} (S_s psi(n+s)) chi(n)^dag        (an N_c x N_c matrix).
// W_s is the average of the k! hop orderings of Tab. off-axis; built level by
// level it obeys W_s(n) = (1/k) sum_{mu in supp s} W_{s - s_mu mu}(n) V_{s_mu mu}(n + s - s_mu mu)
// (grouping the orderings by their last hop), and the adjoint of that
// recursion carries G down the levels:
//   G_{s - s_mu mu} += (1/k) V G_s          (at the same site n),
//   link term  tr[dV X],  X = (1/k) G_s W_{s - s_mu mu},
// where V = U_mu(m) receives K_mu(m) += X and V = U_mu(m - mu)^dag receives
// K_mu(m - mu) += X^dag (m = n + s - s_mu mu), with dS = Re sum tr[dU K].
//
// Kernel 1 (one block per site, one thread per offset): W of the site in
// shared memory (the forward recursion again), M_s from psi(n+s) and chi(n),
// then G level by level from k = 4 down to 1, each level gathering from its
// parents (no atomics: deterministic); every (s, mu) link term X of the site
// goes to a scratch slot.  Kernel 2 (one thread per link): K_mu(m) gathers the
// 54 slots that land on the link -- 27 offsets enter it forward, 27 backward --
// and writes F = P_TA(U K) or G = bc K^dag (force_out of force.cu with C = 0).
// Arithmetic in FP64 for FP64 operators and FP32 otherwise, like the W builder.
#include "bril_dirs.h"
#include "internal.h"
#include "linkalg.cuh"

namespace dgb {

namespace bforce {

__host__ __device__ constexpr int kk(int d) {
    return (d % 3 != 1) + ((d / 3) % 3 != 1) + ((d / 9) % 3 != 1) + (d / 27 != 1);
}
__host__ __device__ constexpr int comp(int d, int mu) {   // s_mu of offset index d
    return mu == 0 ? d % 3 - 1 : mu == 1 ? (d / 3) % 3 - 1 : mu == 2 ? (d / 9) % 3 - 1 : d / 27 - 1;
}
// first scratch slot of offset d: the slots of (d, mu) for mu in supp(s_d), increasing mu
__host__ __device__ constexpr int slot_base(int d) {
    int o = 0;
    for (int j = 0; j < d; ++j) o += kk(j);
    return o;
}
constexpr int kSlots = 216;   // sum over offsets of their hop count
// slot of the link term (d, mu), -1 where offset d does not move along mu:
// a table in constant memory, built at compile time (computing it per call
// took an O(d) loop of integer divisions, which made both force kernels
// integer-bound)
struct SlotTable {
    short slot[81][4];
};
__host__ __device__ constexpr SlotTable make_slot_table() {
    SlotTable t{};
    for (int d = 0; d < 81; ++d) {
        int o = slot_base(d);
        for (int mu = 0; mu < 4; ++mu) t.slot[d][mu] = comp(d, mu) != 0 ? (short)o++ : (short)-1;
    }
    return t;
}
static __constant__ SlotTable kSlotTable = make_slot_table();
__device__ __forceinline__ int slot_of(int d, int mu) { return kSlotTable.slot[d][mu]; }
// x + off on a periodic axis of extent ext, off in {-1, 0, 1}
__device__ __forceinline__ int wrap(int x, int ext) { return x < 0 ? x + ext : (x >= ext ? x - ext : x); }
constexpr int pow3(int mu) { return mu == 0 ? 1 : mu == 1 ? 3 : mu == 2 ? 9 : 27; }

template <int NC, typename E>
using Arith = std::conditional_t<sizeof(E) == 8, double, float>;
template <int NC, typename E>
constexpr size_t site_smem() { return 2 * sizeof(cx<Arith<NC, E>>) * 81 * NC * NC; }

// V_{sign mu}(x) from the operator's phased links: U_mu(x) or U_mu(x - mu)^dag
template <int NC, typename E, typename AB>
__device__ __forceinline__ void hop_link(const E *__restrict__ U, const Lat &g, const int x[4], int mu, int sign,
                                         cx<AB> (&L)[NC][NC]) {
    int y[4] = {x[0], x[1], x[2], x[3]};
    const int ext[4] = {g.nx, g.ny, g.nz, g.nt};
    if (sign < 0) y[mu] = (y[mu] == 0) ? ext[mu] - 1 : y[mu] - 1;
    const long long site = (((long long)y[3] * g.nz + y[2]) * g.ny + y[1]) * g.nx + y[0];
    const E *p = U + 2 * Layout<0>::template mat<NC>(g, site, 4, mu);
    const long long ls = Layout<0>::template mat_stride<NC>(g);
#pragma unroll
    for (int a = 0; a < NC; ++a)
#pragma unroll
        for (int b = 0; b < NC; ++b) {
            const cx<AB> u = ld1<E, AB>(p + 2 * ls * (sign > 0 ? a * NC + b : b * NC + a));
            L[a][b] = sign > 0 ? u : cx<AB>{u.re, -u.im};
        }
}

// (S_s psi)_sigma for one colour and RHS: rho_k sum_mu s_mu (gamma_mu p)_sigma - lambda_k/2 p_sigma,
// gammas of App. A in the chiral basis (the same signed permutations as the stencil)
template <typename A>
__device__ __forceinline__ cx<A> gamma_comp(int mu, int sg, const cx<A> p[4]) {
    // gamma_1 psi = (-i p3, -i p2, i p1, i p0); gamma_2 psi = (-p3, p2, p1, -p0);
    // gamma_3 psi = (-i p2, i p3, i p0, -i p1); gamma_4 psi = (p2, p3, p0, p1)
    switch (mu) {
    case 0: {
        const cx<A> v = p[3 - sg];
        return sg <= 1 ? cx<A>{v.im, -v.re} : cx<A>{-v.im, v.re};
    }
    case 1: {
        const cx<A> v = p[3 - sg];
        return (sg == 0 || sg == 3) ? cx<A>{-v.re, -v.im} : v;
    }
    case 2: {
        const cx<A> v = p[sg ^ 2];
        return (sg == 0 || sg == 3) ? cx<A>{v.im, -v.re} : cx<A>{-v.im, v.re};
    }
    default:
        return p[sg ^ 2];
    }
}

}  // namespace bforce

// Kernel 1: per site n, the 216 link terms X_(s, mu)(n) into scratch[n][slot][NC^2].
template <int NC, typename E, int LAYOUT>
__global__ void __launch_bounds__(96) bril_force_site_kernel(const E *__restrict__ U, const E *__restrict__ psi,
                                                             const E *__restrict__ chi, E *__restrict__ X, Lat g) {
    using AB = bforce::Arith<NC, E>;
    using L = Layout<LAYOUT>;
    extern __shared__ __align__(16) unsigned char bf_smem[];
    auto Ws = reinterpret_cast<cx<AB>(*)[NC * NC]>(bf_smem);
    auto Gs = Ws + 81;
    const long long n = blockIdx.x;
    const int d = threadIdx.x < 81 ? kLevelOrder.d[threadIdx.x] : 81;   // offsets of a level share warps
    const Coord c = site_coords(g, n);
    const int x0[4] = {c.x, c.y, c.z, c.t};
    const int ext[4] = {g.nx, g.ny, g.nz, g.nt};
    int s[4] = {0, 0, 0, 0}, k = -1;
    if (d < 81) {
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) s[mu] = bforce::comp(d, mu);
        k = bforce::kk(d);
    }
    // ---- forward: W_s(n) level by level (W_0 = 1)
    if (k == 0)
        for (int e = 0; e < NC * NC; ++e) Ws[40][e] = cx<AB>{(AB)((e / NC) == (e % NC) ? 1 : 0), (AB)0};
    __syncthreads();
    for (int level = 1; level <= 4; ++level) {
        if (k == level) {
            cx<AB> acc[NC][NC];
            for (int a = 0; a < NC; ++a)
                for (int b = 0; b < NC; ++b) acc[a][b] = cx<AB>{0, 0};
            for (int mu = 0; mu < 4; ++mu) {
                if (s[mu] == 0) continue;
                const int prev = d - s[mu] * bforce::pow3(mu);
                int m[4];
                for (int nu = 0; nu < 4; ++nu) m[nu] = bforce::wrap(x0[nu] + (nu == mu ? 0 : s[nu]), ext[nu]);
                cx<AB> V[NC][NC];
                bforce::hop_link<NC, E, AB>(U, g, m, mu, s[mu], V);
                for (int a = 0; a < NC; ++a)
                    for (int b = 0; b < NC; ++b)
                        for (int q = 0; q < NC; ++q) cmac(acc[a][b], Ws[prev][a * NC + q], V[q][b]);
            }
            const AB inv = (AB)1 / (AB)level;
            for (int a = 0; a < NC; ++a)
                for (int b = 0; b < NC; ++b) Ws[d][a * NC + b] = inv * acc[a][b];
        }
        __syncthreads();
    }
    // ---- G_s = -2 M_s(n),  M_s = sum_{v, spin} (S_s psi(n+s)) chi(n)^dag
    if (k >= 1) {
        const AB rho = (AB)bril::rho(k);
        const AB lam_half = (AB)(0.5 * (double)(1 << (4 - k)) / 64.0);   // lambda_k / 2, lambda = (8,4,2,1)/64
        int m[4];
        for (int nu = 0; nu < 4; ++nu) m[nu] = bforce::wrap(x0[nu] + s[nu], ext[nu]);
        const long long ns = (((long long)m[3] * g.nz + m[2]) * g.ny + m[1]) * g.nx + m[0];
        const long long csd = L::cs_stride(g);
        const long long pb = L::vec(g, ns, NC * 4, 0), cb = L::vec(g, n, NC * 4, 0);
        cx<AB> M[NC][NC];
        for (int a = 0; a < NC; ++a)
            for (int b = 0; b < NC; ++b) M[a][b] = cx<AB>{0, 0};
        for (int v = 0; v < g.nv; ++v) {
            cx<AB> sp[NC][4], ch[NC][4];
#pragma unroll
            for (int a = 0; a < NC; ++a) {
                cx<AB> p[4];
#pragma unroll
                for (int sg = 0; sg < 4; ++sg) {
                    p[sg] = ld1<E, AB>(psi + 2 * (pb + (long long)(a * 4 + sg) * csd + v));
                    ch[a][sg] = ld1<E, AB>(chi + 2 * (cb + (long long)(a * 4 + sg) * csd + v));
                }
#pragma unroll
                for (int sg = 0; sg < 4; ++sg) {
                    cx<AB> f = {-lam_half * p[sg].re, -lam_half * p[sg].im};
#pragma unroll
                    for (int mu = 0; mu < 4; ++mu) {
                        if (s[mu] == 0) continue;
                        const cx<AB> t = bforce::gamma_comp<AB>(mu, sg, p);
                        const AB w = rho * (AB)s[mu];
                        f.re += w * t.re;
                        f.im += w * t.im;
                    }
                    sp[a][sg] = f;
                }
            }
#pragma unroll
            for (int a = 0; a < NC; ++a)
#pragma unroll
                for (int b = 0; b < NC; ++b)
#pragma unroll
                    for (int sg = 0; sg < 4; ++sg) cmac(M[a][b], sp[a][sg], conj(ch[b][sg]));
        }
        for (int a = 0; a < NC; ++a)
            for (int b = 0; b < NC; ++b) Gs[d][a * NC + b] = (AB)-2 * M[a][b];
    }
    __syncthreads();
    // ---- backward, level 4 down to 1
    for (int level = 4; level >= 1; --level) {
        if (k == level) {
            // link terms X = (1/k) G_s W_{s - s_mu mu} of this offset
            const AB inv = (AB)1 / (AB)level;
            for (int mu = 0; mu < 4; ++mu) {
                if (s[mu] == 0) continue;
                const int prev = d - s[mu] * bforce::pow3(mu);
                E *o = X + 2 * (((long long)n * bforce::kSlots + bforce::slot_of(d, mu)) * NC * NC);
                for (int a = 0; a < NC; ++a)
                    for (int b = 0; b < NC; ++b) {
                        cx<AB> t = {0, 0};
                        for (int q = 0; q < NC; ++q) cmac(t, Gs[d][a * NC + q], Ws[prev][q * NC + b]);
                        o[2 * (a * NC + b)] = from_acc<E, AB>(inv * t.re);
                        o[2 * (a * NC + b) + 1] = from_acc<E, AB>(inv * t.im);
                    }
            }
        }
        __syncthreads();
        if (level > 1 && k == level - 1) {
            // G_p += (1/level) V_{sign mu}(n + p) G_{p + sign mu}  over the parents of p
            const AB inv = (AB)1 / (AB)level;
            int m[4];
            for (int nu = 0; nu < 4; ++nu) m[nu] = bforce::wrap(x0[nu] + s[nu], ext[nu]);
            cx<AB> acc[NC][NC];
            for (int a = 0; a < NC; ++a)
                for (int b = 0; b < NC; ++b) acc[a][b] = Gs[d][a * NC + b];
            for (int mu = 0; mu < 4; ++mu) {
                if (s[mu] != 0) continue;
                for (int sign = -1; sign <= 1; sign += 2) {
                    const int child = d + sign * bforce::pow3(mu);
                    cx<AB> V[NC][NC];
                    bforce::hop_link<NC, E, AB>(U, g, m, mu, sign, V);
                    for (int a = 0; a < NC; ++a)
                        for (int b = 0; b < NC; ++b) {
                            cx<AB> t = {0, 0};
                            for (int q = 0; q < NC; ++q) cmac(t, V[a][q], Gs[child][q * NC + b]);
                            acc[a][b] = acc[a][b] + inv * t;
                        }
                }
            }
            for (int a = 0; a < NC; ++a)
                for (int b = 0; b < NC; ++b) Gs[d][a * NC + b] = acc[a][b];
        }
        __syncthreads();
    }
}

// Kernel 2: K_mu(m) from the 54 slots landing on link (m, mu), then F or G.
template <int NC, typename E, int LAYOUT>
__global__ void bril_force_link_kernel(const E *__restrict__ U, const E *__restrict__ X, E *__restrict__ out, Lat g,
                                       int bc0, int bc1, int bc2, int bc3, int mode) {
    using A = typename Acc<E>::T;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= g.V * 4) return;
    const long long m = tid / 4;
    const int mu = (int)(tid % 4);
    const Coord c = site_coords(g, m);
    const int xm[4] = {c.x, c.y, c.z, c.t};
    const int ext[4] = {g.nx, g.ny, g.nz, g.nt};
    cx<A> K[NC][NC];
    for (int a = 0; a < NC; ++a)
        for (int b = 0; b < NC; ++b) K[a][b] = cx<A>{0, 0};
    for (int d = 0; d < 81; ++d) {
        const int smu = bforce::comp(d, mu);
        if (smu == 0) continue;
        // forward hop (s_mu = +1): n = m + mu - s;  backward hop (s_mu = -1): n = m - s
        int nn[4];
#pragma unroll
        for (int nu = 0; nu < 4; ++nu) {
            const int sn = bforce::comp(d, nu);
            const int off = (smu > 0 && nu == mu) ? 1 - sn : -sn;
            nn[nu] = bforce::wrap(xm[nu] + off, ext[nu]);
        }
        const long long n = (((long long)nn[3] * g.nz + nn[2]) * g.ny + nn[1]) * g.nx + nn[0];
        const E *x = X + 2 * ((n * bforce::kSlots + bforce::slot_of(d, mu)) * NC * NC);
        for (int a = 0; a < NC; ++a)
            for (int b = 0; b < NC; ++b) {
                const cx<A> v = ld1<E, A>(x + 2 * (smu > 0 ? a * NC + b : b * NC + a));
                K[a][b] = K[a][b] + (smu > 0 ? v : conj(v));
            }
    }
    E *o = out + 2 * (tid * NC * NC);
    if (mode == 1) {   // G = bc K^dag for the caller's unphased links
        const int bcm = mu == 0 ? bc0 : mu == 1 ? bc1 : mu == 2 ? bc2 : bc3;
        const A ph = (xm[mu] == ext[mu] - 1) ? (A)bcm : (A)1;
        for (int a = 0; a < NC; ++a)
            for (int b = 0; b < NC; ++b) {
                o[2 * (a * NC + b)] = from_acc<E, A>(ph * K[b][a].re);
                o[2 * (a * NC + b) + 1] = from_acc<E, A>(-ph * K[b][a].im);
            }
        return;
    }
    // F = P_TA(U K), U the phased link
    cx<A> Lk[NC][NC], M[NC][NC];
    load_mat_s<NC, E, A>(U + 2 * Layout<0>::template mat<NC>(g, m, 4, mu), Layout<0>::template mat_stride<NC>(g), Lk);
    for (int a = 0; a < NC; ++a)
        for (int b = 0; b < NC; ++b) {
            cx<A> acc = {0, 0};
            for (int q = 0; q < NC; ++q) cmac(acc, Lk[a][q], K[q][b]);
            M[a][b] = acc;
        }
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

// Brillouin force: scratch of 216 link terms per site, owned by the operator
// (allocated on first use, freed with it).
int launch_bril_force(dirac_op *op, const void *psi, const void *chi, void *out, int mode, cudaStream_t s) {
    const size_t need = (size_t)op->V * bforce::kSlots * op->nc * op->nc * 2 * elem_bytes(op->prec);
    if (op->force_ws_bytes < need) {
        cudaFree(op->force_ws);
        op->force_ws = nullptr;
        op->force_ws_bytes = 0;
        if (cudaMalloc(&op->force_ws, need) != cudaSuccess) {
            cudaGetLastError();
            op->force_ws = nullptr;
            return DIRAC_ERR_OOM;
        }
        op->force_ws_bytes = need;
    }
    return dispatch_prec(op->prec, [&](auto tag) {
        using E = std::remove_pointer_t<decltype(tag)>;
        if constexpr (sizeof(E) == 2) {
            return (int)DIRAC_ERR_UNSUPPORTED_PREC;
        } else {
            return dispatch_nc(op->nc, [&](auto ncc) {
                constexpr int NC = decltype(ncc)::value;
                return dispatch_layout(op->geom.layout, [&](auto lyc) {
                    constexpr int LAYOUT = decltype(lyc)::value;
                    constexpr size_t smem = bforce::site_smem<NC, E>();
                    if constexpr (smem > 48 * 1024) {
                        const int rc = cuda_check(cudaFuncSetAttribute(bril_force_site_kernel<NC, E, LAYOUT>,
                                                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                                       (int)smem),
                                                  "bril_force_site_kernel shared memory");
                        if (rc) return rc;
                    }
                    bril_force_site_kernel<NC, E, LAYOUT><<<(unsigned)op->V, 96, smem, s>>>(
                        (const E *)op->links, (const E *)psi, (const E *)chi, (E *)op->force_ws, op->lat);
                    int rc = launch_check("bril_force_site_kernel");
                    if (rc) return rc;
                    const int *bc = op->geom.bc;
                    bril_force_link_kernel<NC, E, LAYOUT><<<grid_for(op->V * 4, 128), 128, 0, s>>>(
                        (const E *)op->links, (const E *)op->force_ws, (E *)out, op->lat, bc[0], bc[1], bc[2], bc[3],
                        mode);
                    return launch_check("bril_force_link_kernel");
                });
            });
        }
    });
}

}  // namespace dgb
