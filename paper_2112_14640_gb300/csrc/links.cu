// links.cu -- gauge-field preparation done once per field:
//  * phase_links: the operator's own copy of U in its storage precision with
//    the boundary phase bc[mu] folded into U_mu(n) where n_mu = N_mu - 1;
//  * build_w: the 80 off-centre Brillouin links of Tab. off-axis,
//      W_s(n) = (1/k!) sum over the k! minimal paths n -> n+s of the ordered
//               products of signed links V_{+mu}(m) = U_mu(m), V_{-mu}(m) = U_mu(m-mu)^dag.
//    Grouping the paths by their last hop sigma gives the recursion
//      W_s(n) = (1/k) sum_{mu: s_mu != 0} W_{s - s_mu mu}(n) V_{s_mu mu}(n + s - s_mu mu),
//    evaluated level by level (k = 1..4) in shared memory, one thread block
//    per site, in FP64 for FP64 operators and FP32 otherwise; the result is
//    stored in the link precision;
//  * build_clover: the clover term of Eq. (def_clov) in the block form of
//    clover.cuh, from the clover-leaf field strength
//      F_mu,nu(n) = (Q_mu,nu(n) - Q_mu,nu(n)^dag) / (8i),
//    Q the sum of the four plaquettes of the (mu,nu) plane with a corner at
//    n, all traversed the same way (mu-step first, then nu-step);
//  * stout_smear: the fat links V the paper builds its operators and F
//    from (Sec. 2, App. F), steps of Morningstar-Peardon stout smearing.
#include "bril_dirs.h"
#include "internal.h"
#include "linkalg.cuh"

namespace dgb {

struct Phases {
    int bc[4];
};


template <typename UE, typename E>
__global__ void phase_links_kernel(const UE *__restrict__ U, E *__restrict__ out, Lat g, Phases ph, int nc,
                                   int layout) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;   // (site, mu)
    if (tid >= g.V * 4) return;
    const long long n = tid / 4;
    const int mu = (int)(tid % 4);
    const Coord c = site_coords(g, n);
    const int coord = mu == 0 ? c.x : mu == 1 ? c.y : mu == 2 ? c.z : c.t;
    const int ext = mu == 0 ? g.nx : mu == 1 ? g.ny : mu == 2 ? g.nz : g.nt;
    const double f = (coord == ext - 1) ? (double)ph.bc[mu] : 1.0;
    const int per = nc * nc;
    for (int e = 0; e < per; ++e) {
        cx<double> u = ld_u(U, tid * per + e);
        // blocks of 32 sites, [mu][a][b][site % 32] within (common.cuh, link_index)
        const long long o = link_index(n, 4, per, mu, e);
        out[2 * o] = from_acc<E, double>(f * u.re);
        out[2 * o + 1] = from_acc<E, double>(f * u.im);
    }
}

// signed link V_{sign mu}(m) with boundary phase, in the arithmetic type AB
template <int NC, typename UE, typename AB>
__device__ __forceinline__ void signed_link(const UE *__restrict__ U, const Lat &g, const Phases &ph,
                                            const int x[4], int mu, int sign, cx<AB> (&L)[NC][NC]) {
    const int ext[4] = {g.nx, g.ny, g.nz, g.nt};
    int y[4] = {x[0], x[1], x[2], x[3]};
    if (sign < 0) y[mu] = (y[mu] == 0) ? ext[mu] - 1 : y[mu] - 1;
    const long long site = (((long long)y[3] * g.nz + y[2]) * g.ny + y[1]) * g.nx + y[0];
    const double f = (y[mu] == ext[mu] - 1) ? (double)ph.bc[mu] : 1.0;
    const long long base = (site * 4 + mu) * NC * NC;
#pragma unroll
    for (int a = 0; a < NC; ++a)
#pragma unroll
        for (int b = 0; b < NC; ++b) {
            cx<double> u = ld_u(U, base + (sign > 0 ? a * NC + b : b * NC + a));
            L[a][b] = sign > 0 ? cx<AB>{(AB)(f * u.re), (AB)(f * u.im)} : cx<AB>{(AB)(f * u.re), (AB)(-f * u.im)};
        }
}

// W in FP64 for FP64 links, in FP32 otherwise (FP32 links carry 24 bits; the
// four levels add a few FP32 roundings, and FP64 arithmetic is slow here).
template <int NC, typename E>
using WArith = std::conditional_t<sizeof(E) == 8, double, float>;
// shared memory of build_w_kernel: the 81 W_s of one site
template <int NC, typename E>
constexpr size_t build_w_smem() { return sizeof(cx<WArith<NC, E>>) * 81 * NC * NC; }

template <int NC, typename UE, typename E>
__global__ void __launch_bounds__(96) build_w_kernel(const UE *__restrict__ U, E *__restrict__ W, Lat g, Phases ph) {
    using AB = WArith<NC, E>;
    // dynamic: 81 N_c^2 complex numbers exceed the static 48 KB for N_c >= 7 in FP64
    extern __shared__ __align__(16) unsigned char w_smem[];
    auto Ws = reinterpret_cast<cx<AB>(*)[NC * NC]>(w_smem);
    const long long n = blockIdx.x;
    const int dir = threadIdx.x < 81 ? kLevelOrder.d[threadIdx.x] : 81;   // offsets of a level share warps
    const Coord c = site_coords(g, n);
    const int x0[4] = {c.x, c.y, c.z, c.t};
    const int ext[4] = {g.nx, g.ny, g.nz, g.nt};
    int s[4] = {0, 0, 0, 0}, k = 0;
    if (dir < 81) {
        s[0] = dir % 3 - 1;
        s[1] = (dir / 3) % 3 - 1;
        s[2] = (dir / 9) % 3 - 1;
        s[3] = dir / 27 - 1;
        k = (s[0] != 0) + (s[1] != 0) + (s[2] != 0) + (s[3] != 0);
        if (k == 0)
            for (int a = 0; a < NC; ++a)
                for (int b = 0; b < NC; ++b) Ws[40][a * NC + b] = cx<AB>{(AB)(a == b ? 1 : 0), (AB)0};
    }
    const int pow3[4] = {1, 3, 9, 27};
    // the last hop of the term along mu starts at n + s - s_mu mu
    auto last_hop = [&](int mu, cx<AB> (&L)[NC][NC]) {
        int m[4];
        for (int nu = 0; nu < 4; ++nu) {
            int v = x0[nu] + (nu == mu ? 0 : s[nu]);
            m[nu] = (v + ext[nu]) % ext[nu];
        }
        signed_link<NC, UE, AB>(U, g, ph, m, mu, s[mu], L);
    };
    // N_c <= 4: every link this offset needs (one per axis it moves along) is
    // requested before the first level, so that the four levels do not each
    // wait for their own loads
    constexpr bool kPreload = NC <= kMaxNcSmall;
    cx<AB> Lpre[kPreload ? 4 : 1][NC][NC];   // by axis: compile-time indices keep them in registers
    if constexpr (kPreload) {
        if (dir < 81) {
#pragma unroll
            for (int mu = 0; mu < 4; ++mu)
                if (s[mu] != 0) last_hop(mu, Lpre[mu]);
        }
    }
    __syncthreads();   // the identity at the centre feeds level 1
    for (int level = 1; level <= 4; ++level) {
        if (dir < 81 && k == level) {
            cx<AB> acc[NC][NC];
            for (int a = 0; a < NC; ++a)
                for (int b = 0; b < NC; ++b) acc[a][b] = cx<AB>{0, 0};
#pragma unroll
            for (int mu = 0; mu < 4; ++mu) {
                if (s[mu] == 0) continue;
                const int prev = dir - s[mu] * pow3[mu];   // offset s - s_mu mu
                cx<AB> Lrt[NC][NC];
                if constexpr (!kPreload) last_hop(mu, Lrt);
                const cx<AB>(&L)[NC][NC] = kPreload ? Lpre[kPreload ? mu : 0] : Lrt;
                for (int a = 0; a < NC; ++a)
                    for (int b = 0; b < NC; ++b)
                        for (int q = 0; q < NC; ++q) cmac(acc[a][b], Ws[prev][a * NC + q], L[q][b]);
            }
            const AB inv = (AB)1 / (AB)level;
            for (int a = 0; a < NC; ++a)
                for (int b = 0; b < NC; ++b) Ws[dir][a * NC + b] = inv * acc[a][b];
        }
        __syncthreads();
    }
    if (dir < 81 && dir != 40) {
        // stored as rho_k s_lead W_s at index q (bril_dirs.h)
        double scale;
        const int q = bril::store_index(s, &scale);
        for (int e = 0; e < NC * NC; ++e) {
            // [site][q][a][b] for either vector layout
            const long long o = bril::w_index(q, e, n, NC);
            W[2 * o] = from_acc<E, double>(scale * (double)Ws[dir][e].re);
            W[2 * o + 1] = from_acc<E, double>(scale * (double)Ws[dir][e].im);
        }
    }
}

// The stored W~ back to W_s in the public order d = (st+1)*27 + (sz+1)*9 +
// (sy+1)*3 + (sx+1), centre left out, in the operator's layout and link precision.
template <typename E>
__global__ void unpack_w_kernel(const E *__restrict__ Wst, E *__restrict__ out, Lat g, int nc, int layout) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;   // (site, dirp)
    if (tid >= g.V * 80) return;
    const long long n = tid / 80;
    const int dirp = (int)(tid % 80);
    const int dir = dirp < 40 ? dirp : dirp + 1;
    const int s[4] = {dir % 3 - 1, (dir / 3) % 3 - 1, (dir / 9) % 3 - 1, dir / 27 - 1};
    double scale;
    const int q = bril::store_index(s, &scale);
    const int per = nc * nc;
    for (int e = 0; e < per; ++e) {
        const long long i = bril::w_index(q, e, n, nc);
        const long long o = layout == 0 ? (n * 80 + dirp) * per + e : ((long long)dirp * per + e) * g.V + n;
        using A = typename Acc<E>::T;
        out[2 * o] = from_acc<E, double>((double)to_acc<E>(Wst[2 * i]) / scale);
        out[2 * o + 1] = from_acc<E, double>((double)to_acc<E>(Wst[2 * i + 1]) / scale);
    }
}

int launch_unpack_w(const dirac_op *op, void *out, cudaStream_t s) {
    return dispatch_prec(link_prec(op), [&](auto tag) {
        using E = std::remove_pointer_t<decltype(tag)>;
        const long long threads = op->V * 80;
        unpack_w_kernel<E><<<grid_for(threads, 128), 128, 0, s>>>((const E *)op->w, (E *)out, op->lat, op->nc,
                                                                  op->geom.layout);
        return launch_check("unpack_w_kernel");
    });
}


static Phases phases_of(const dirac_op *op) {
    Phases ph;
    for (int m = 0; m < 4; ++m) ph.bc[m] = op->geom.bc[m];
    return ph;
}

int launch_phase_links(dirac_op *op, const void *U, dirac_prec u_prec, cudaStream_t s) {
    return dispatch_uprec(u_prec, [&](auto utag) {
        using UE = std::remove_pointer_t<decltype(utag)>;
        return dispatch_prec(link_prec(op), [&](auto tag) {
            using E = std::remove_pointer_t<decltype(tag)>;
            const long long threads = op->V * 4;
            phase_links_kernel<UE, E><<<grid_for(threads, 128), 128, 0, s>>>((const UE *)U, (E *)op->links,
                                                                            op->lat, phases_of(op), op->nc,
                                                                            op->geom.layout);
            return launch_check("phase_links_kernel");
        });
    });
}

int launch_build_w(dirac_op *op, const void *U, dirac_prec u_prec, cudaStream_t s) {
    return dispatch_uprec(u_prec, [&](auto utag) {
        using UE = std::remove_pointer_t<decltype(utag)>;
        return dispatch_prec(link_prec(op), [&](auto tag) {
            using E = std::remove_pointer_t<decltype(tag)>;
            return dispatch_nc<big_nc_ok<E>()>(op->nc, [&](auto ncc) {
                constexpr int NC = decltype(ncc)::value;
                constexpr size_t smem = build_w_smem<NC, E>();
                if constexpr (smem > 48 * 1024) {
                    const int rc = cuda_check(cudaFuncSetAttribute(build_w_kernel<NC, UE, E>,
                                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                                   (int)smem),
                                              "build_w_kernel shared memory");
                    if (rc) return rc;
                }
                build_w_kernel<NC, UE, E><<<(unsigned)op->V, 96, smem, s>>>((const UE *)U, (E *)op->w, op->lat,
                                                                          phases_of(op));
                return launch_check("build_w_kernel");
            });
        });
    });
}

// ------------------------------------------------------------ clover term


// F_mu,nu at site x0 from the four leaves (+mu,+nu), (+nu,-mu), (-mu,-nu),
// (-nu,+mu); the leaf (a, b) is V_a(n) V_b(n+a) V_-a(n+a+b) V_-b(n+b).
template <int NC, typename UE, typename AB>
__device__ void field_strength(const UE *__restrict__ U, const Lat &g, const Phases &ph, const int x0[4], int mu,
                               int nu, cx<AB> (&F)[NC][NC]) {
    const int ext[4] = {g.nx, g.ny, g.nz, g.nt};
    const int st[4][4] = {{mu, 1, nu, 1}, {nu, 1, mu, -1}, {mu, -1, nu, -1}, {nu, -1, mu, 1}};
    cx<AB> Q[NC][NC];
#pragma unroll
    for (int a = 0; a < NC; ++a)
#pragma unroll
        for (int b = 0; b < NC; ++b) Q[a][b] = cx<AB>{0, 0};
    for (int l = 0; l < 4; ++l) {
        const int am = st[l][0], as = st[l][1], bm = st[l][2], bs = st[l][3];
        int xa[4] = {x0[0], x0[1], x0[2], x0[3]};
        step(xa, ext, am, as);
        int xab[4] = {xa[0], xa[1], xa[2], xa[3]};
        step(xab, ext, bm, bs);
        int xb[4] = {x0[0], x0[1], x0[2], x0[3]};
        step(xb, ext, bm, bs);
        cx<AB> P[NC][NC], L[NC][NC], T[NC][NC];
        signed_link<NC, UE, AB>(U, g, ph, x0, am, as, P);
        signed_link<NC, UE, AB>(U, g, ph, xa, bm, bs, L);
        mat_mul<NC, AB>(P, L, T);
        signed_link<NC, UE, AB>(U, g, ph, xab, am, -as, L);
        mat_mul<NC, AB>(T, L, P);
        signed_link<NC, UE, AB>(U, g, ph, xb, bm, -bs, L);
        mat_mul<NC, AB>(P, L, T);
#pragma unroll
        for (int a = 0; a < NC; ++a)
#pragma unroll
            for (int b = 0; b < NC; ++b) Q[a][b] = Q[a][b] + T[a][b];
    }
    // (Q - Q^dag) / (8i) = -i (Q - Q^dag) / 8
#pragma unroll
    for (int a = 0; a < NC; ++a)
#pragma unroll
        for (int b = 0; b < NC; ++b) {
            const cx<AB> d = {Q[a][b].re - Q[b][a].re, Q[a][b].im + Q[b][a].im};
            F[a][b] = cx<AB>{d.im / (AB)8, -d.re / (AB)8};
        }
}

// One thread per (site, block k = 2 chi + w): block A (w = 0) of chirality chi
// needs the planes (1,2), (3,4); block B (w = 1) the planes (1,4), (2,3),
// (1,3), (2,4) (clover.cuh).  FP64 arithmetic for FP64 storage, FP32 otherwise.
template <int NC, typename UE, typename E>
__global__ void __launch_bounds__(128) build_clover_kernel(const UE *__restrict__ U, E *__restrict__ out, Lat g,
                                                           Phases ph, double csw, int layout) {
    using AB = std::conditional_t<sizeof(E) == 8, double, float>;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= g.V * 4) return;
    const long long n = tid / 4;
    const int k = (int)(tid % 4), chi = k >> 1, w = k & 1;
    const AB e = chi == 0 ? (AB)1 : (AB)-1;
    const Coord c = site_coords(g, n);
    const int x0[4] = {c.x, c.y, c.z, c.t};
    // (plane, complex coefficient) pairs of the block, planes as (mu, nu) 0-based
    int planes[4][2];
    cx<AB> coef[4];
    int np;
    if (w == 0) {   // -F_12 + e F_34
        np = 2;
        planes[0][0] = 0, planes[0][1] = 1, coef[0] = cx<AB>{-1, 0};
        planes[1][0] = 2, planes[1][1] = 3, coef[1] = cx<AB>{e, 0};
    } else {        // e F_14 - F_23 - i F_13 - i e F_24
        np = 4;
        planes[0][0] = 0, planes[0][1] = 3, coef[0] = cx<AB>{e, 0};
        planes[1][0] = 1, planes[1][1] = 2, coef[1] = cx<AB>{-1, 0};
        planes[2][0] = 0, planes[2][1] = 2, coef[2] = cx<AB>{0, -1};
        planes[3][0] = 1, planes[3][1] = 3, coef[3] = cx<AB>{0, -e};
    }
    cx<AB> acc[NC][NC];
#pragma unroll
    for (int a = 0; a < NC; ++a)
#pragma unroll
        for (int b = 0; b < NC; ++b) acc[a][b] = cx<AB>{0, 0};
    for (int i = 0; i < np; ++i) {
        cx<AB> F[NC][NC];
        field_strength<NC, UE, AB>(U, g, ph, x0, planes[i][0], planes[i][1], F);
#pragma unroll
        for (int a = 0; a < NC; ++a)
#pragma unroll
            for (int b = 0; b < NC; ++b) cmac(acc[a][b], coef[i], F[a][b]);
    }
    const double f = -0.5 * csw;
    const int per = NC * NC;
#pragma unroll
    for (int a = 0; a < NC; ++a)
#pragma unroll
        for (int b = 0; b < NC; ++b) {
            const int el = a * NC + b;
            // the links' layout (common.cuh, link_index)
            const long long o = link_index(n, 4, per, k, el);
            out[2 * o] = from_acc<E, double>(f * (double)acc[a][b].re);
            out[2 * o + 1] = from_acc<E, double>(f * (double)acc[a][b].im);
        }
}

int launch_build_clover(dirac_op *op, const void *V, dirac_prec v_prec, cudaStream_t s) {
    return dispatch_uprec(v_prec, [&](auto utag) {
        using UE = std::remove_pointer_t<decltype(utag)>;
        return dispatch_prec(link_prec(op), [&](auto tag) {
            using E = std::remove_pointer_t<decltype(tag)>;
            return dispatch_nc<big_nc_ok<E>()>(op->nc, [&](auto ncc) {
                constexpr int NC = decltype(ncc)::value;
                const long long threads = op->V * 4;
                // closed loops do not see the boundary phases: leave them out
                Phases none;
                for (int m = 0; m < 4; ++m) none.bc[m] = 1;
                build_clover_kernel<NC, UE, E><<<grid_for(threads, 128), 128, 0, s>>>(
                    (const UE *)V, (E *)op->clover, op->lat, none, op->csw, op->geom.layout);
                return launch_check("build_clover_kernel");
            });
        });
    });
}

template <typename S, typename D>
__global__ void convert_scalars_kernel(const S *__restrict__ src, D *__restrict__ dst, long long count) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) dst[i] = from_acc<D, typename Acc<S>::T>(to_acc<S>(src[i]));
}

static int convert_array(const void *src, dirac_prec sp, void *dst, dirac_prec dp, long long count, cudaStream_t s) {
    return dispatch_prec(sp, [&](auto stag) {
        using S = std::remove_pointer_t<decltype(stag)>;
        return dispatch_prec(dp, [&](auto dtag) {
            using D = std::remove_pointer_t<decltype(dtag)>;
            convert_scalars_kernel<S, D><<<grid_for(count, 256), 256, 0, s>>>((const S *)src, (D *)dst, count);
            return launch_check("convert_scalars_kernel");
        });
    });
}

int launch_convert_links(const dirac_op *src, dirac_op *dst, cudaStream_t s) {
    long long n = link_sites(src->V) * 4 * src->nc * src->nc * 2;
    int rc = convert_array(src->links, link_prec(src), dst->links, link_prec(dst), n, s);
    if (rc) return rc;
    if (src->w) {
        // same order, scale and layout, element by element
        n = src->V * 80 * src->nc * src->nc * 2;
        rc = convert_array(src->w, link_prec(src), dst->w, link_prec(dst), n, s);
    }
    if (!rc && src->clover) {
        n = link_sites(src->V) * 4 * src->nc * src->nc * 2;
        rc = convert_array(src->clover, link_prec(src), dst->clover, link_prec(dst), n, s);
    }
    return rc;
}

}  // namespace dgb
