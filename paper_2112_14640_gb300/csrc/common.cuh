// common.cuh -- device-side building blocks shared by the stencil, BLAS-1
// and solver kernels: complex arithmetic in the accumulation type,
// precision-generic vectorised loads/stores of interleaved complex data, and
// lattice index arithmetic (site n = ((t*Nz + z)*Ny + y)*Nx + x).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/dirac.h"

namespace dgb {

// ------------------------------------------------------------------ complex
template <typename A>
struct cx {
    A re, im;
};

template <typename A>
__host__ __device__ __forceinline__ cx<A> mk(A r, A i) { return cx<A>{r, i}; }
template <typename A>
__device__ __forceinline__ cx<A> operator+(cx<A> a, cx<A> b) { return {a.re + b.re, a.im + b.im}; }
template <typename A>
__device__ __forceinline__ cx<A> operator-(cx<A> a, cx<A> b) { return {a.re - b.re, a.im - b.im}; }
template <typename A>
__device__ __forceinline__ cx<A> operator*(A s, cx<A> a) { return {s * a.re, s * a.im}; }
template <typename A>
__device__ __forceinline__ cx<A> conj(cx<A> a) { return {a.re, -a.im}; }
// i * a
template <typename A>
__device__ __forceinline__ cx<A> times_i(cx<A> a) { return {-a.im, a.re}; }
// acc += a * b (complex), written as four FMAs
template <typename A>
__device__ __forceinline__ void cmac(cx<A> &acc, cx<A> a, cx<A> b) {
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(-a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(a.im, b.re, acc.im);
}
// acc += conj(a) * b
template <typename A>
__device__ __forceinline__ void cmac_conj(cx<A> &acc, cx<A> a, cx<A> b) {
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(-a.im, b.re, acc.im);
}
template <typename A>
__device__ __forceinline__ cx<A> cmul(cx<A> a, cx<A> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// acc += s * a (real s)
template <typename A>
__device__ __forceinline__ void rmac(cx<A> &acc, A s, cx<A> a) {
    acc.re = fma(s, a.re, acc.re);
    acc.im = fma(s, a.im, acc.im);
}

// -------------------------------------------------------- storage elements
template <typename E> struct Acc { using T = float; };
template <> struct Acc<double> { using T = double; };

template <typename E> __device__ __forceinline__ typename Acc<E>::T to_acc(E e);
template <> __device__ __forceinline__ double to_acc<double>(double e) { return e; }
template <> __device__ __forceinline__ float to_acc<float>(float e) { return e; }
template <> __device__ __forceinline__ float to_acc<__nv_bfloat16>(__nv_bfloat16 e) { return __bfloat162float(e); }
template <> __device__ __forceinline__ float to_acc<__half>(__half e) { return __half2float(e); }

template <typename E, typename A> __device__ __forceinline__ E from_acc(A a);
template <> __device__ __forceinline__ double from_acc<double, double>(double a) { return a; }
template <> __device__ __forceinline__ float from_acc<float, float>(float a) { return a; }
template <> __device__ __forceinline__ __nv_bfloat16 from_acc<__nv_bfloat16, float>(float a) { return __float2bfloat16_rn(a); }
template <> __device__ __forceinline__ __half from_acc<__half, float>(float a) { return __float2half_rn(a); }
// conversions between accumulation types (used by precision casts)
template <> __device__ __forceinline__ float from_acc<float, double>(double a) { return (float)a; }
template <> __device__ __forceinline__ double from_acc<double, float>(float a) { return (double)a; }
template <> __device__ __forceinline__ __nv_bfloat16 from_acc<__nv_bfloat16, double>(double a) { return __double2bfloat16(a); }
template <> __device__ __forceinline__ __half from_acc<__half, double>(double a) { return __double2half(a); }

template <int BYTES> struct Raw;
template <> struct Raw<16> { using T = uint4; };
template <> struct Raw<8> { using T = uint2; };
template <> struct Raw<4> { using T = unsigned int; };

// Load N consecutive complex numbers starting at element pointer p (2N
// elements), converting to the accumulation type.  Uses 16-byte (or smaller)
// vector loads; p must be aligned to min(16, 2*N*sizeof(E)) bytes.
template <typename E, int N, typename A = typename Acc<E>::T>
__device__ __forceinline__ void load_cx(const E *__restrict__ p, cx<A> *out) {
    constexpr int BYTES = 2 * N * (int)sizeof(E);
    if constexpr (BYTES <= 16) {
        using R = typename Raw<BYTES>::T;
        R raw = __ldg(reinterpret_cast<const R *>(p));
        E e[2 * N];
        __builtin_memcpy(e, &raw, BYTES);
#pragma unroll
        for (int i = 0; i < N; ++i) out[i] = cx<A>{(A)to_acc<E>(e[2 * i]), (A)to_acc<E>(e[2 * i + 1])};
    } else {
        constexpr int PER = 16 / (2 * (int)sizeof(E));
#pragma unroll
        for (int k = 0; k < N / PER; ++k) load_cx<E, PER, A>(p + 2 * PER * k, out + PER * k);
    }
}

template <typename E, int N, typename A>
__device__ __forceinline__ void store_cx(E *__restrict__ p, const cx<A> *in) {
    constexpr int BYTES = 2 * N * (int)sizeof(E);
    if constexpr (BYTES <= 16) {
        using R = typename Raw<BYTES>::T;
        E e[2 * N];
#pragma unroll
        for (int i = 0; i < N; ++i) {
            e[2 * i] = from_acc<E, A>(in[i].re);
            e[2 * i + 1] = from_acc<E, A>(in[i].im);
        }
        R raw;
        __builtin_memcpy(&raw, e, BYTES);
        *reinterpret_cast<R *>(p) = raw;
    } else {
        constexpr int PER = 16 / (2 * (int)sizeof(E));
#pragma unroll
        for (int k = 0; k < N / PER; ++k) store_cx<E, PER, A>(p + 2 * PER * k, in + PER * k);
    }
}

// Single complex load without vector width requirements (links, W links).
template <typename E, typename A = typename Acc<E>::T>
__device__ __forceinline__ cx<A> ld1(const E *__restrict__ p) {
    if constexpr (sizeof(E) == 8) {
        double2 d = __ldg(reinterpret_cast<const double2 *>(p));
        return cx<A>{(A)d.x, (A)d.y};
    } else if constexpr (sizeof(E) == 4) {
        float2 f = __ldg(reinterpret_cast<const float2 *>(p));
        return cx<A>{(A)f.x, (A)f.y};
    } else {
        cx<A> r;
        load_cx<E, 1, A>(p, &r);
        return r;
    }
}

// Load an NC x NC colour matrix (row-major, complex) into registers.
template <int NC, typename E, typename A>
__device__ __forceinline__ void load_mat(const E *__restrict__ p, cx<A> (&M)[NC][NC]) {
#pragma unroll
    for (int a = 0; a < NC; ++a)
#pragma unroll
        for (int b = 0; b < NC; ++b) M[a][b] = ld1<E, A>(p + 2 * (a * NC + b));
}

// --------------------------------------------------------------- geometry
struct Lat {
    int nx, ny, nz, nt;
    int nv;
    long long V;
    // output sites a stencil launch covers: n0 .. n0 + nsites - 1 (the whole
    // lattice unless a pipelined host apply works slab by slab)
    long long n0, nsites;
};

struct Coord {
    int x, y, z, t;
};

// Site coordinates with 32-bit unsigned division: volumes are at most 2^31
// sites (checked when an operator is created), and a 64-bit division is a
// long instruction sequence that every stencil thread would pay six times.
__device__ __forceinline__ Coord site_coords(const Lat &g, long long n) {
    Coord c;
    const unsigned u = (unsigned)n;
    unsigned r = u / (unsigned)g.nx;
    c.x = (int)(u - r * (unsigned)g.nx);
    unsigned r2 = r / (unsigned)g.ny;
    c.y = (int)(r - r2 * (unsigned)g.ny);
    r = r2 / (unsigned)g.nz;
    c.z = (int)(r2 - r * (unsigned)g.nz);
    c.t = (int)r;
    return c;
}

// Thread index -> (output site offset i, RHS chunk j) of a stencil launch,
// with 32-bit division whenever the index fits.
__device__ __forceinline__ void split_tid(long long tid, int nchunk, long long &i, int &j) {
    if (tid < 0xFFFFFFFFLL) {
        const unsigned t = (unsigned)tid, q = t / (unsigned)nchunk;
        i = q;
        j = (int)(t - q * (unsigned)nchunk);
    } else {
        i = tid / nchunk;
        j = (int)(tid - i * nchunk);
    }
}

// Site index of the neighbour n + sign * mu-hat (periodic wrap).
__device__ __forceinline__ long long neighbour(const Lat &g, long long n, const Coord &c, int mu, int sign) {
    long long stride;
    int coord, extent;
    switch (mu) {
    case 0: stride = 1; coord = c.x; extent = g.nx; break;
    case 1: stride = g.nx; coord = c.y; extent = g.ny; break;
    case 2: stride = (long long)g.nx * g.ny; coord = c.z; extent = g.nz; break;
    default: stride = (long long)g.nx * g.ny * g.nz; coord = c.t; extent = g.nt; break;
    }
    if (sign > 0) return (coord == extent - 1) ? n - (long long)(extent - 1) * stride : n + stride;
    return (coord == 0) ? n + (long long)(extent - 1) * stride : n - stride;
}

// ------------------------------------------------------------- layouts
// Index arithmetic of the two vector layouts (in complex numbers).  ncs is the
// number of internal components per site (N_c*4 or N_c), cs one of them.
//   OUTER: ((site * ncs + cs) * nv + v)      INNER: ((cs * V + site) * nv + v)
// Links and clover blocks, element e of matrix k (k = mu or block) of site n,
// for either vector layout and N_c <= 4: blocks of kLinkBlock consecutive
// sites, within a block [k][e][n % kLinkBlock] (link_index).  Consecutive sites' elements are
// adjacent, so the link loads of a warp coalesce whether its threads cover 32
// sites (one RHS) or a few sites with many RHS each, and one block's matrices
// stay within a few KB.  (Measured at 16^3x32, FP32: [k][e][site] over the
// whole field, D_W 0.105 ms at N_v = 12; [site][k][e], 0.097 ms at N_v = 12
// but 35-45% slower D_W and D_S at N_v = 1.)  Buffers are padded to a whole
// number of blocks (link_sites).
constexpr int kLinkBlockLog2 = 5, kLinkBlock = 1 << kLinkBlockLog2;
__host__ __device__ __forceinline__ long long link_sites(long long V) {
    return (V + kLinkBlock - 1) >> kLinkBlockLog2 << kLinkBlockLog2;
}
// Above N_c = 4 (per = N_c^2 > 16) the stencils read a link one row at a
// time, one RHS per thread: there a site's matrices stay contiguous
// ([site][k][a][b], element stride 1), so that a row is one run of N_c
// complex numbers (32-site blocks measured 15-35% slower for D_W and D_S at
// N_c = 6, 8).
__host__ __device__ constexpr int link_stride(int per) { return per > 16 ? 1 : kLinkBlock; }
// site >= 0: shifts instead of signed division
__host__ __device__ __forceinline__ long long link_index(long long site, int nk, int per, int k, int e) {
    if (per > 16) return (site * nk + k) * per + e;
    return (((site >> kLinkBlockLog2) * nk * per + (long long)k * per + e) << kLinkBlockLog2) +
           (site & (kLinkBlock - 1));
}
template <int LAYOUT>
struct Layout {
    static __host__ __device__ __forceinline__ long long vec(const Lat &g, long long site, int ncs, int cs) {
        if constexpr (LAYOUT == 0) return (site * ncs + cs) * (long long)g.nv;
        else return ((long long)cs * g.V + site) * g.nv;
    }
    // distance (in complex numbers) between consecutive components cs of one site
    static __host__ __device__ __forceinline__ long long cs_stride(const Lat &g) {
        if constexpr (LAYOUT == 0) return g.nv;
        else return g.V * g.nv;
    }
    // element 0 of matrix k of site `site` (nk matrices per site)
    template <int NC>
    static __host__ __device__ __forceinline__ long long mat(const Lat &, long long site, int nk, int k) {
        return link_index(site, nk, NC * NC, k, 0);
    }
    // distance between consecutive matrix elements
    template <int NC>
    static __host__ __device__ __forceinline__ long long mat_stride(const Lat &) { return link_stride(NC * NC); }
};

// NC x NC matrix whose elements are `stride` complex numbers apart.
template <int NC, typename E, typename A>
__device__ __forceinline__ void load_mat_s(const E *__restrict__ p, long long stride, cx<A> (&M)[NC][NC]) {
#pragma unroll
    for (int a = 0; a < NC; ++a)
#pragma unroll
        for (int b = 0; b < NC; ++b) M[a][b] = ld1<E, A>(p + 2 * stride * (a * NC + b));
}

// Element type for each storage precision.
template <int P> struct Elem;
template <> struct Elem<DIRAC_F64> { using T = double; };
template <> struct Elem<DIRAC_F32> { using T = float; };
template <> struct Elem<DIRAC_BF16> { using T = __nv_bfloat16; };
template <> struct Elem<DIRAC_F16> { using T = __half; };

}  // namespace dgb
