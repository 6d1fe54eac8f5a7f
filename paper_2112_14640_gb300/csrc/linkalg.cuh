// linkalg.cuh -- colour-matrix helpers shared by the link kernels (links.cu:
// phases, W links, clover term) and the stout kernels (stout.cu): element
// loads in FP64, matrix products, the periodic coordinate step, and exp of an
// N x N matrix by scaling and squaring of its Taylor series.
#pragma once
#include "internal.h"

namespace dgb {

// The 81 offsets d = (st+1)*27 + (sz+1)*9 + (sy+1)*3 + (sx+1) of the
// 3^4 hypercube, ordered by level (the number of axes an offset moves
// along: 8, 24, 32, 16 of them) with the centre last.  Kernels that run
// one thread per offset and work level by level map thread t to offset
// kLevelOrder.d[t], so that each level occupies whole warps (threads 0-31:
// levels 1 and 2, 32-63: level 3, 64-79: level 4) instead of a few lanes of
// every warp.
struct LevelOrder {
    int d[81];
};
__host__ __device__ constexpr LevelOrder make_level_order() {
    LevelOrder t{};
    int i = 0;
    for (int k = 1; k <= 4; ++k)
        for (int d = 0; d < 81; ++d)
            if ((d % 3 != 1) + ((d / 3) % 3 != 1) + ((d / 9) % 3 != 1) + (d / 27 != 1) == k) t.d[i++] = d;
    t.d[i] = 40;
    return t;
}
static __constant__ LevelOrder kLevelOrder = make_level_order();


template <typename UE>
__device__ __forceinline__ cx<double> ld_u(const UE *U, long long idx) {
    return cx<double>{(double)U[2 * idx], (double)U[2 * idx + 1]};
}

template <typename F>
inline int dispatch_uprec(dirac_prec p, F &&f) {
    if (p == DIRAC_F64) return f((double *)nullptr);
    if (p == DIRAC_F32) return f((float *)nullptr);
    return DIRAC_ERR_UNSUPPORTED_PREC;
}

// fully unrolled for N_c <= 4; the outer loops stay loops above that (code
// size and compile time: the W builder, clover and stout kernels hold several
// such products per thread)
template <int NC, typename AB>
__device__ __forceinline__ void mat_mul(const cx<AB> (&X)[NC][NC], const cx<AB> (&Y)[NC][NC], cx<AB> (&Z)[NC][NC]) {
#pragma unroll(NC <= 4 ? NC : 1)
    for (int a = 0; a < NC; ++a)
#pragma unroll(NC <= 4 ? NC : 1)
        for (int b = 0; b < NC; ++b) {
            cx<AB> t = {0, 0};
#pragma unroll
            for (int q = 0; q < NC; ++q) cmac(t, X[a][q], Y[q][b]);
            Z[a][b] = t;
        }
}

__device__ __forceinline__ void step(int (&x)[4], const int ext[4], int mu, int sign) {
    x[mu] = sign > 0 ? (x[mu] + 1 == ext[mu] ? 0 : x[mu] + 1) : (x[mu] == 0 ? ext[mu] - 1 : x[mu] - 1);
}

template <int NC, typename UE>
__device__ __forceinline__ void load_link(const UE *__restrict__ U, const Lat &g, const int x[4], int mu,
                                          cx<double> (&L)[NC][NC]) {
    const long long site = (((long long)x[3] * g.nz + x[2]) * g.ny + x[1]) * g.nx + x[0];
    const long long base = (site * 4 + mu) * NC * NC;
#pragma unroll
    for (int a = 0; a < NC; ++a)
#pragma unroll
        for (int b = 0; b < NC; ++b) L[a][b] = ld_u(U, base + a * NC + b);
}

template <int NC>
__device__ __forceinline__ void mul_nn(const cx<double> (&X)[NC][NC], const cx<double> (&Y)[NC][NC],
                                       cx<double> (&Z)[NC][NC]) {
    mat_mul<NC, double>(X, Y, Z);
}

// Z = X Y^dag
template <int NC>
__device__ __forceinline__ void mul_nd(const cx<double> (&X)[NC][NC], const cx<double> (&Y)[NC][NC],
                                       cx<double> (&Z)[NC][NC]) {
#pragma unroll
    for (int a = 0; a < NC; ++a)
#pragma unroll
        for (int b = 0; b < NC; ++b) {
            cx<double> t = {0, 0};
#pragma unroll
            for (int q = 0; q < NC; ++q) cmac_conj(t, Y[b][q], X[a][q]);
            Z[a][b] = t;
        }
}

// Z = X^dag Y
template <int NC>
__device__ __forceinline__ void mul_dn(const cx<double> (&X)[NC][NC], const cx<double> (&Y)[NC][NC],
                                       cx<double> (&Z)[NC][NC]) {
#pragma unroll
    for (int a = 0; a < NC; ++a)
#pragma unroll
        for (int b = 0; b < NC; ++b) {
            cx<double> t = {0, 0};
#pragma unroll
            for (int q = 0; q < NC; ++q) cmac_conj(t, X[q][a], Y[q][b]);
            Z[a][b] = t;
        }
}

template <int NC>
__device__ void expm_taylor(cx<double> (&X)[NC][NC], cx<double> (&E)[NC][NC]) {
    double nrm = 0;
    for (int a = 0; a < NC; ++a) {
        double r = 0;
        for (int b = 0; b < NC; ++b) r += sqrt(X[a][b].re * X[a][b].re + X[a][b].im * X[a][b].im);
        nrm = fmax(nrm, r);
    }
    int sq = 0;
    while (nrm > 0.25 && sq < 40) {
        nrm *= 0.5;
        ++sq;
    }
    const double f = ldexp(1.0, -sq);
    cx<double> T[NC][NC], P[NC][NC];
    for (int a = 0; a < NC; ++a)
        for (int b = 0; b < NC; ++b) {
            X[a][b] = cx<double>{f * X[a][b].re, f * X[a][b].im};
            T[a][b] = cx<double>{a == b ? 1.0 : 0.0, 0.0};
            E[a][b] = T[a][b];
        }
#pragma unroll 1
    for (int k = 1; k <= 30; ++k) {
        mat_mul<NC, double>(T, X, P);   // T_k = T_{k-1} X / k
        double tn = 0, en = 0;
        for (int a = 0; a < NC; ++a)
            for (int b = 0; b < NC; ++b) {
                T[a][b] = cx<double>{P[a][b].re / k, P[a][b].im / k};
                E[a][b] = E[a][b] + T[a][b];
                tn = fmax(tn, fabs(T[a][b].re) + fabs(T[a][b].im));
                en = fmax(en, fabs(E[a][b].re) + fabs(E[a][b].im));
            }
        if (tn <= 1e-17 * en) break;
    }
#pragma unroll 1
    for (int i = 0; i < sq; ++i) {
        mat_mul<NC, double>(E, E, P);
        for (int a = 0; a < NC; ++a)
            for (int b = 0; b < NC; ++b) E[a][b] = P[a][b];
    }
}


}  // namespace dgb
