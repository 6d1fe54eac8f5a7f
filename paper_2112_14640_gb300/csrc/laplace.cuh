// laplace.cuh -- multi-RHS Laplace operators A = -1/2 Lap + m^2/2 (Secs. 6
// and 7; the paper's wlap, blap, wsuv, bsuv routines of App. F):
//   Eq. (app_wlap): (A psi)(n) = (4 + m^2/2) psi(n)
//        - 1/2 sum_mu [ U_mu(n) psi(n+mu) + U_mu(n-mu)^dag psi(n-mu) ]
//   Eq. (app_blap): (A psi)(n) = (m^2/2 - lambda_0/2) psi(n) - 1/2 sum_{s != 0} lambda_k W_s(n) psi(n+s)
// acting trivially on NS spin components per colour (NS = 4: Wilson-type
// vectors, NS = 1: colour-only vectors).  A is hermitian: no dagger variant.
//
// Same thread mapping as the Dirac stencils (thread <-> site, VR consecutive
// right-hand sides; write-once register accumulator).  The Brillouin
// Laplacian reads the operator's stored W~_q = rho_k s_lead W_s (bril_dirs.h),
// per site in visiting order, and weighs each with -c_k s_lead, which is
// -lambda_k/2 on W_s; offsets and weights come from a table in constant
// memory (one broadcast read per offset, uniform over the warp).
#pragma once
#include "bril_dirs.h"
#include "internal.h"

namespace dgb {
namespace bril {

// The offsets in storage order with the weight of the Brillouin Laplacian on
// the stored W~: -lambda_k/2 W_s = -c_k s_lead W~_q (Eq. app_blap).
struct OffsetTable {
    signed char s[80][4];
    double lap[80];
};
__host__ __device__ constexpr OffsetTable make_offset_table() {
    OffsetTable t{};
    int q = 0;
    for (int m = 1; m < 16; ++m) {
        const int k = popc4(m);
        for (int b = 0; b < (1 << k); ++b, ++q) {
            int j = 0;
            for (int mu = 0; mu < 4; ++mu) {
                t.s[q][mu] = 0;
                if ((m >> mu) & 1) {
                    t.s[q][mu] = ((b >> j) & 1) ? -1 : 1;
                    ++j;
                }
            }
            t.lap[q] = -c_lambda(k) * (double)t.s[q][lead_axis(m)];
        }
    }
    return t;
}

}  // namespace bril

static __constant__ bril::OffsetTable kLapOffsets = bril::make_offset_table();

// Whether a hop multiplies its weight into the N_c x N_c matrix once (N_c^2
// complex scalings) instead of into each of the NS VR N_c products (one real
// multiply-add per complex component): worth it when NS VR > N_c.
template <int NC, int NS, int VR>
constexpr bool fold_weight() { return NS * VR > NC; }

// acc[c][s] += f L psi(m) (or f L^dag psi(m)) for every spin component s
template <int NC, int NS, int VR, bool DAG, typename E, typename A>
__device__ __forceinline__ void lap_hop(cx<A> (&acc)[NC][NS][VR], const cx<A> (&Lin)[NC][NC],
                                        const E *__restrict__ psi, long long cs_stride, A f) {
    constexpr bool FOLD = fold_weight<NC, NS, VR>();
    cx<A> Lf[NC][NC];
    if constexpr (FOLD) {
#pragma unroll
        for (int a = 0; a < NC; ++a)
#pragma unroll
            for (int b = 0; b < NC; ++b) Lf[a][b] = cx<A>{f * Lin[a][b].re, f * Lin[a][b].im};
    }
    const cx<A>(*L)[NC] = FOLD ? (const cx<A>(*)[NC])Lf : Lin;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        if constexpr (FOLD) {
            // one colour component of the neighbour at a time (VR complex
            // numbers in registers, not N_c VR)
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                cx<A> pk[VR];
                load_cx<E, VR, A>(psi + 2 * (k * NS + s) * cs_stride, pk);
#pragma unroll
                for (int c = 0; c < NC; ++c)
#pragma unroll
                    for (int v = 0; v < VR; ++v) {
                        if constexpr (DAG) cmac_conj(acc[c][s][v], L[k][c], pk[v]);
                        else cmac(acc[c][s][v], L[c][k], pk[v]);
                    }
            }
        } else {
            cx<A> p[NC][VR];
#pragma unroll
            for (int k = 0; k < NC; ++k) load_cx<E, VR, A>(psi + 2 * (k * NS + s) * cs_stride, p[k]);
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
                    rmac(acc[c][s][v], f, t);
                }
        }
    }
}

template <int NC, int NS, int VR, int LAYOUT, typename E, typename A>
__device__ __forceinline__ void lap_write(const E *__restrict__ in, E *__restrict__ out, const Lat &g,
                                          long long n, int j, A centre, const cx<A> (&acc)[NC][NS][VR]) {
    using L = Layout<LAYOUT>;
    const long long cs = L::cs_stride(g);
    const long long base = 2 * (L::vec(g, n, NC * NS, 0) + (long long)j * VR);
#pragma unroll
    for (int a = 0; a < NC; ++a)
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            cx<A> p[VR], o[VR];
            const long long off = base + 2LL * (a * NS + s) * cs;
            load_cx<E, VR, A>(in + off, p);
#pragma unroll
            for (int v = 0; v < VR; ++v) o[v] = centre * p[v] + acc[a][s][v];
            store_cx<E, VR, A>(out + off, o);
        }
}

// Eq. (app_wlap): centre = 4 + m^2/2, each hop weighted -1/2
template <int NC, int NS, int VR, typename E, int MINB, int LAYOUT>
__global__ void __launch_bounds__(stencil_max_threads(MINB), (MINB > 1 ? 1 : 0))
    wlap_kernel(const E *__restrict__ U, const E *__restrict__ in, E *__restrict__ out, Lat g,
                typename Acc<E>::T centre) {
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
    const long long cs = L::cs_stride(g), ls = L::template mat_stride<NC>(g);

    cx<A> acc[NC][NS][VR];
#pragma unroll
    for (int a = 0; a < NC; ++a)
#pragma unroll
        for (int s = 0; s < NS; ++s)
#pragma unroll
            for (int v = 0; v < VR; ++v) acc[a][s][v] = cx<A>{0, 0};
    const A mhalf = (A)-0.5;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        const long long fw = neighbour(g, n, c, mu, +1);
        const long long bw = neighbour(g, n, c, mu, -1);
        cx<A> Lm[NC][NC];
        load_mat_s<NC, E, A>(U + 2 * L::template mat<NC>(g, n, 4, mu), ls, Lm);
        lap_hop<NC, NS, VR, false>(acc, Lm, in + 2 * (L::vec(g, fw, NC * NS, 0) + (long long)j * VR), cs, mhalf);
        load_mat_s<NC, E, A>(U + 2 * L::template mat<NC>(g, bw, 4, mu), ls, Lm);
        lap_hop<NC, NS, VR, true>(acc, Lm, in + 2 * (L::vec(g, bw, NC * NS, 0) + (long long)j * VR), cs, mhalf);
    }
    lap_write<NC, NS, VR, LAYOUT, E, A>(in, out, g, n, j, centre, acc);
}

// Eq. (app_blap): centre = m^2/2 - lambda_0/2, offset q weighted kLapOffsets.lap[q] on W~_q
template <int NC, int NS, int VR, typename E, int MINB, int LAYOUT>
__global__ void __launch_bounds__(stencil_max_threads(MINB), (MINB > 1 ? 1 : 0))
    blap_kernel(const E *__restrict__ W, const E *__restrict__ in, E *__restrict__ out, Lat g,
                typename Acc<E>::T centre) {
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
    const long long cs = L::cs_stride(g);
    // site-index steps of +1 / -1 along each axis, with the periodic wrap
    // (32-bit: volumes are below 2^31 sites)
    int dp[4], dm[4];
    {
        const int co[4] = {c.x, c.y, c.z, c.t};
        const int ext[4] = {g.nx, g.ny, g.nz, g.nt};
        int stride = 1;
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            dp[mu] = (co[mu] == ext[mu] - 1 ? -(ext[mu] - 1) : 1) * stride;
            dm[mu] = (co[mu] == 0 ? ext[mu] - 1 : -1) * stride;
            stride *= ext[mu];
        }
    }
    cx<A> acc[NC][NS][VR];
#pragma unroll
    for (int a = 0; a < NC; ++a)
#pragma unroll
        for (int s = 0; s < NS; ++s)
#pragma unroll
            for (int v = 0; v < VR; ++v) acc[a][s][v] = cx<A>{0, 0};
    // W~ of one site contiguous in visiting order (either vector layout)
    const E *wp = W + 2LL * n * 80 * NC * NC;
    const E *inj = in + 2LL * j * VR;
    auto hop = [&](int q, const cx<A>(&Wm)[NC][NC]) {
        int m = (int)n;
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            const int sm = kLapOffsets.s[q][mu];
            m += sm > 0 ? dp[mu] : (sm < 0 ? dm[mu] : 0);
        }
        lap_hop<NC, NS, VR, false>(acc, Wm, inj + 2 * L::vec(g, (long long)m, NC * NS, 0), cs,
                                   (A)kLapOffsets.lap[q]);
    };
    if constexpr (NC <= kMaxNcSmall) {
        // two offsets per trip: the W~ of the next offset is loaded while the
        // current one is applied, the two buffers swapping roles (80 is even)
        cx<A> Wa[NC][NC], Wb[NC][NC];
        load_mat<NC, E, A>(wp, Wa);
#pragma unroll 1
        for (int q = 0; q < 80; q += 2) {
            load_mat<NC, E, A>(wp + 2 * (q + 1) * NC * NC, Wb);
            hop(q, Wa);
            if (q + 2 < 80) load_mat<NC, E, A>(wp + 2 * (q + 2) * NC * NC, Wa);
            hop(q + 1, Wb);
        }
    } else {
        // large N_c: one N_c x N_c buffer (the register file holds no second one)
#pragma unroll 1
        for (int q = 0; q < 80; ++q) {
            cx<A> Wm[NC][NC];
            load_mat<NC, E, A>(wp + 2 * q * NC * NC, Wm);
            hop(q, Wm);
        }
    }
    lap_write<NC, NS, VR, LAYOUT, E, A>(in, out, g, n, j, centre, acc);
}

template <typename E, int LAYOUT>
int launch_laplace_v(const dirac_op *op, const void *in, void *out, double m, cudaStream_t s) {
    int vr, minb, block;
    launch_variant(op, vr, minb, block);
    using A = typename Acc<E>::T;
    const bool bril = uses_w(op->kind);
    const double centre = bril ? 0.5 * m * m + 240.0 / 128.0 : 4.0 + 0.5 * m * m;
    return dispatch_nc<big_nc_ok<E>()>(op->nc, [&](auto ncc) {
        constexpr int NC = decltype(ncc)::value;
        return dispatch_vr(vr, [&](auto vrc) {
            constexpr int VR = decltype(vrc)::value;
            if constexpr (!vr_compiled<NC>(VR)) return (int)DIRAC_ERR_INVALID_ARG;
            else return dispatch_minb<NC>(minb, [&](auto mbc) {
                constexpr int MINB = decltype(mbc)::value;
                const long long threads = op->lat.nsites * (op->nv / VR);
                auto go = [&](auto nsc) {
                    constexpr int NS = decltype(nsc)::value;
                    if (bril)
                        blap_kernel<NC, NS, VR, E, MINB, LAYOUT><<<grid_for(threads, block), block, 0, s>>>(
                            (const E *)op->w, (const E *)in, (E *)out, op->lat, (A)centre);
                    else
                        wlap_kernel<NC, NS, VR, E, MINB, LAYOUT><<<grid_for(threads, block), block, 0, s>>>(
                            (const E *)op->links, (const E *)in, (E *)out, op->lat, (A)centre);
                    return launch_check(bril ? "blap_kernel" : "wlap_kernel");
                };
                return spins_of(op->kind) == 4 ? go(std::integral_constant<int, 4>{})
                                               : go(std::integral_constant<int, 1>{});
            });
        });
    });
}

}  // namespace dgb
