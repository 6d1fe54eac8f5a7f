// stout.cu -- stout smearing of a gauge field and the chain rule of a link
// derivative through it (dirac_stout_smear, dirac_stout_backward).
#include "internal.h"
#include "linkalg.cuh"

namespace dgb {

// ------------------------------------------------------------ stout smearing
// One step, one thread per link (n, mu), FP64 arithmetic for either storage:
//   C = rho sum_{nu != mu} [U_nu(n) U_mu(n+nu) U_nu(n+mu)^dag + U_nu(n-nu)^dag U_mu(n-nu) U_nu(n-nu+mu)],
//   Omega = C U_mu(n)^dag,  Q = (i/2)(Omega^dag - Omega) - (i/2N) Tr(Omega^dag - Omega),
//   U'_mu(n) = exp(iQ) U_mu(n).
// exp(iQ) by scaling and squaring of the Taylor series (Moler and Van Loan):
// X = iQ / 2^s with ||X||_inf <= 1/4, the series summed until a term falls
// below 1e-17 of the partial sum (at most 30 terms), then squared s times;
// valid for every N_c.

// Staple sum Cs = rho C and X = iQ (traceless anti-hermitian) of link (x0, mu)
// for one stout step; A receives U_mu(x0).
template <int NC, typename UE>
__device__ void stout_parts(const UE *__restrict__ U, const Lat &g, const int x0[4], int mu, double rho,
                            cx<double> (&Cs)[NC][NC], cx<double> (&X)[NC][NC], cx<double> (&A)[NC][NC]) {
    const int ext[4] = {g.nx, g.ny, g.nz, g.nt};
    cx<double> B[NC][NC], T[NC][NC];
    for (int a = 0; a < NC; ++a)
        for (int b = 0; b < NC; ++b) Cs[a][b] = cx<double>{0, 0};
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
        int xm[4] = {x0[0], x0[1], x0[2], x0[3]}, xn[4] = {x0[0], x0[1], x0[2], x0[3]};
        step(xm, ext, mu, +1);   // n + mu
        step(xn, ext, nu, +1);   // n + nu
        // forward staple U_nu(n) U_mu(n+nu) U_nu(n+mu)^dag
        load_link<NC, UE>(U, g, x0, nu, A);
        load_link<NC, UE>(U, g, xn, mu, B);
        mul_nn<NC>(A, B, T);
        load_link<NC, UE>(U, g, xm, nu, A);
        mul_nd<NC>(T, A, B);
        for (int a = 0; a < NC; ++a)
            for (int b = 0; b < NC; ++b) Cs[a][b] = Cs[a][b] + B[a][b];
        // backward staple U_nu(n-nu)^dag U_mu(n-nu) U_nu(n-nu+mu)
        int xb[4] = {x0[0], x0[1], x0[2], x0[3]};
        step(xb, ext, nu, -1);   // n - nu
        int xbm[4] = {xb[0], xb[1], xb[2], xb[3]};
        step(xbm, ext, mu, +1);  // n - nu + mu
        load_link<NC, UE>(U, g, xb, nu, A);
        load_link<NC, UE>(U, g, xb, mu, B);
        mul_dn<NC>(A, B, T);
        load_link<NC, UE>(U, g, xbm, nu, A);
        mul_nn<NC>(T, A, B);
        for (int a = 0; a < NC; ++a)
            for (int b = 0; b < NC; ++b) Cs[a][b] = Cs[a][b] + B[a][b];
    }
    for (int a = 0; a < NC; ++a)
        for (int b = 0; b < NC; ++b) Cs[a][b] = cx<double>{rho * Cs[a][b].re, rho * Cs[a][b].im};
    // Omega = Cs U_mu(n)^dag
    load_link<NC, UE>(U, g, x0, mu, A);
    mul_nd<NC>(Cs, A, T);
    // X = iQ = -(1/2) D + (1/2N) Tr(D), D = Omega^dag - Omega: traceless anti-hermitian
    for (int a = 0; a < NC; ++a)
        for (int b = 0; b < NC; ++b) {
            // D = Omega^dag - Omega, element (a, b) = conj(Om[b][a]) - Om[a][b]
            const cx<double> d = {T[b][a].re - T[a][b].re, -T[b][a].im - T[a][b].im};
            X[a][b] = cx<double>{-0.5 * d.re, -0.5 * d.im};
        }
    // subtract Tr(-D/2)/N from the diagonal
    cx<double> trx = {0, 0};
    for (int a = 0; a < NC; ++a) trx = trx + X[a][a];
    for (int a = 0; a < NC; ++a) X[a][a] = X[a][a] - cx<double>{trx.re / NC, trx.im / NC};
}

template <int NC, typename UE>
__global__ void __launch_bounds__(128) stout_step_kernel(const UE *__restrict__ U, UE *__restrict__ out, Lat g,
                                                         double rho) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= g.V * 4) return;
    const long long n = tid / 4;
    const int mu = (int)(tid % 4);
    const Coord c = site_coords(g, n);
    const int x0[4] = {c.x, c.y, c.z, c.t};
    cx<double> Cs[NC][NC], A[NC][NC], B[NC][NC], T[NC][NC];
    stout_parts<NC, UE>(U, g, x0, mu, rho, Cs, B, A);
    expm_taylor<NC>(B, T);
    mul_nn<NC>(T, A, B);
    const long long base = tid * NC * NC;
    for (int a = 0; a < NC; ++a)
        for (int b = 0; b < NC; ++b) {
            out[2 * (base + a * NC + b)] = (UE)B[a][b].re;
            out[2 * (base + a * NC + b) + 1] = (UE)B[a][b].im;
        }
}

// ------------------------------------------- chain rule through stout smearing
// The derivative in the form dS = Re sum tr[dV Sigma] (Sigma = G^dag of the
// dirac_force GRAD convention) is carried from the output V' = exp(iQ) U of
// a step to its input U:
//   Sigma_U = Sigma' e^{iQ} - Cs^dag Xi  + the staple terms of Y = U^dag Xi,
//   Lambda = L(iQ, U Sigma'), the Frechet derivative of exp at iQ applied to
//            U Sigma' (tr[d e^{iQ} U Sigma'] = tr[i dQ Lambda]), here the
//            upper-right block of exp([[iQ, U Sigma'], [0, iQ]]),
//   Xi = the anti-hermitian part of Lambda - tr(Lambda)/N.
// Kernel 1 (one thread per link): the own terms and Y.  Kernel 2 (one thread
// per link): gathers the 18 staple terms of the links whose staples contain
// it (3 directions x 6 positions), deterministic, no atomics.

template <int NC, typename UE>
__global__ void __launch_bounds__(128) stout_back_own_kernel(const UE *__restrict__ U, const double *__restrict__ Sig,
                                                             double *__restrict__ SigOut, double *__restrict__ Y, Lat g,
                                                             double rho) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= g.V * 4) return;
    const long long n = tid / 4;
    const int mu = (int)(tid % 4);
    const Coord c = site_coords(g, n);
    const int x0[4] = {c.x, c.y, c.z, c.t};
    cx<double> Cs[NC][NC], X[NC][NC], Uo[NC][NC], E[NC][NC], S[NC][NC], T[NC][NC];
    stout_parts<NC, UE>(U, g, x0, mu, rho, Cs, X, Uo);
    const long long base = tid * NC * NC;
    for (int a = 0; a < NC; ++a)
        for (int b = 0; b < NC; ++b) S[a][b] = cx<double>{Sig[2 * (base + a * NC + b)], Sig[2 * (base + a * NC + b) + 1]};
    // block matrix [[iQ, U Sigma'], [0, iQ]]: its exponential carries e^{iQ} and Lambda
    cx<double> Z[2 * NC][2 * NC], EZ[2 * NC][2 * NC];
    mul_nn<NC>(Uo, S, T);
    for (int a = 0; a < 2 * NC; ++a)
        for (int b = 0; b < 2 * NC; ++b) {
            if (a < NC && b < NC) Z[a][b] = X[a][b];
            else if (a >= NC && b >= NC) Z[a][b] = X[a - NC][b - NC];
            else if (a < NC) Z[a][b] = T[a][b - NC];
            else Z[a][b] = cx<double>{0, 0};
        }
    expm_taylor<2 * NC>(Z, EZ);
    cx<double> L[NC][NC];
    for (int a = 0; a < NC; ++a)
        for (int b = 0; b < NC; ++b) {
            E[a][b] = EZ[a][b];
            L[a][b] = EZ[a][b + NC];
        }
    cx<double> tr = {0, 0};
    for (int a = 0; a < NC; ++a) tr = tr + L[a][a];
    for (int a = 0; a < NC; ++a) L[a][a] = L[a][a] - cx<double>{tr.re / NC, tr.im / NC};
    cx<double> Xi[NC][NC];
    for (int a = 0; a < NC; ++a)
        for (int b = 0; b < NC; ++b)   // (L - L^dag) / 2
            Xi[a][b] = cx<double>{0.5 * (L[a][b].re - L[b][a].re), 0.5 * (L[a][b].im + L[b][a].im)};
    // own terms: Sigma' e^{iQ} - Cs^dag Xi
    mul_nn<NC>(S, E, T);
    mul_dn<NC>(Cs, Xi, X);
    for (int a = 0; a < NC; ++a)
        for (int b = 0; b < NC; ++b) {
            SigOut[2 * (base + a * NC + b)] = T[a][b].re - X[a][b].re;
            SigOut[2 * (base + a * NC + b) + 1] = T[a][b].im - X[a][b].im;
        }
    // Y = U^dag Xi
    mul_dn<NC>(Uo, Xi, T);
    for (int a = 0; a < NC; ++a)
        for (int b = 0; b < NC; ++b) {
            Y[2 * (base + a * NC + b)] = T[a][b].re;
            Y[2 * (base + a * NC + b) + 1] = T[a][b].im;
        }
}

template <int NC>
__device__ __forceinline__ void load_d(const double *__restrict__ P, const Lat &g, const int x[4], int mu,
                                       cx<double> (&M)[NC][NC]) {
    const long long site = (((long long)x[3] * g.nz + x[2]) * g.ny + x[1]) * g.nx + x[0];
    const long long base = (site * 4 + mu) * NC * NC;
    for (int a = 0; a < NC; ++a)
        for (int b = 0; b < NC; ++b) M[a][b] = cx<double>{P[2 * (base + a * NC + b)], P[2 * (base + a * NC + b) + 1]};
}

// acc += rho * (X1 X2 X3) or rho * (X1 X2 X3)^dag
template <int NC>
__device__ __forceinline__ void add3(cx<double> (&acc)[NC][NC], const cx<double> (&X1)[NC][NC],
                                     const cx<double> (&X2)[NC][NC], const cx<double> (&X3)[NC][NC], double rho,
                                     bool dag) {
    cx<double> T[NC][NC], P[NC][NC];
    mat_mul<NC, double>(X1, X2, T);
    mat_mul<NC, double>(T, X3, P);
    for (int a = 0; a < NC; ++a)
        for (int b = 0; b < NC; ++b) {
            const cx<double> v = dag ? cx<double>{P[b][a].re, -P[b][a].im} : P[a][b];
            acc[a][b] = acc[a][b] + cx<double>{rho * v.re, rho * v.im};
        }
}

template <int NC>
__device__ __forceinline__ void dagm(const cx<double> (&X)[NC][NC], cx<double> (&Z)[NC][NC]) {
    for (int a = 0; a < NC; ++a)
        for (int b = 0; b < NC; ++b) Z[a][b] = cx<double>{X[b][a].re, -X[b][a].im};
}

template <int NC, typename UE>
__global__ void __launch_bounds__(128) stout_back_staple_kernel(const UE *__restrict__ U, const double *__restrict__ Y,
                                                                double *__restrict__ SigOut, Lat g, double rho) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;   // link (y, alpha)
    if (tid >= g.V * 4) return;
    const long long n = tid / 4;
    const int al = (int)(tid % 4);
    const Coord c = site_coords(g, n);
    const int y[4] = {c.x, c.y, c.z, c.t};
    const int ext[4] = {g.nx, g.ny, g.nz, g.nt};
    cx<double> acc[NC][NC], A1[NC][NC], A2[NC][NC], A3[NC][NC], T[NC][NC];
    for (int a = 0; a < NC; ++a)
        for (int b = 0; b < NC; ++b) acc[a][b] = cx<double>{0, 0};
    for (int be = 0; be < 4; ++be) {
        if (be == al) continue;
        int ya[4] = {y[0], y[1], y[2], y[3]}, yb[4] = {y[0], y[1], y[2], y[3]}, ymb[4] = {y[0], y[1], y[2], y[3]};
        step(ya, ext, al, +1);   // y + alpha
        step(yb, ext, be, +1);   // y + beta
        step(ymb, ext, be, -1);  // y - beta
        int ymba[4] = {ymb[0], ymb[1], ymb[2], ymb[3]};
        step(ymba, ext, al, +1); // y - beta + alpha
        // T1: rho U_be(y+al) U_al(y+be)^dag Y_be(y)
        load_link<NC, UE>(U, g, ya, be, A1);
        load_link<NC, UE>(U, g, yb, al, T);
        dagm<NC>(T, A2);
        load_d<NC>(Y, g, y, be, A3);
        add3<NC>(acc, A1, A2, A3, rho, false);
        // T2: rho U_be(y-be+al)^dag Y_al(y-be) U_be(y-be)
        load_link<NC, UE>(U, g, ymba, be, T);
        dagm<NC>(T, A1);
        load_d<NC>(Y, g, ymb, al, A2);
        load_link<NC, UE>(U, g, ymb, be, A3);
        add3<NC>(acc, A1, A2, A3, rho, false);
        // T3: rho (Y_be(y-be) U_al(y-be) U_be(y-be+al))^dag
        load_d<NC>(Y, g, ymb, be, A1);
        load_link<NC, UE>(U, g, ymb, al, A2);
        load_link<NC, UE>(U, g, ymba, be, A3);
        add3<NC>(acc, A1, A2, A3, rho, true);
        // T4: rho (U_be(y) U_al(y+be) Y_be(y+al))^dag
        load_link<NC, UE>(U, g, y, be, A1);
        load_link<NC, UE>(U, g, yb, al, A2);
        load_d<NC>(Y, g, ya, be, A3);
        add3<NC>(acc, A1, A2, A3, rho, true);
        // T5: rho U_be(y+al) Y_al(y+be) U_be(y)^dag
        load_link<NC, UE>(U, g, ya, be, A1);
        load_d<NC>(Y, g, yb, al, A2);
        load_link<NC, UE>(U, g, y, be, T);
        dagm<NC>(T, A3);
        add3<NC>(acc, A1, A2, A3, rho, false);
        // T6: rho Y_be(y+al-be) U_al(y-be)^dag U_be(y-be)
        load_d<NC>(Y, g, ymba, be, A1);
        load_link<NC, UE>(U, g, ymb, al, T);
        dagm<NC>(T, A2);
        load_link<NC, UE>(U, g, ymb, be, A3);
        add3<NC>(acc, A1, A2, A3, rho, false);
    }
    const long long base = tid * NC * NC;
    for (int a = 0; a < NC; ++a)
        for (int b = 0; b < NC; ++b) {
            SigOut[2 * (base + a * NC + b)] += acc[a][b].re;
            SigOut[2 * (base + a * NC + b) + 1] += acc[a][b].im;
        }
}

// per-link dagger between storage precision S and FP64 (either direction)
template <int NC, typename S, typename D>
__global__ void dagger_links_kernel(const S *__restrict__ in, D *__restrict__ out, long long nlinks) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= nlinks) return;
    const long long base = tid * NC * NC;
    for (int a = 0; a < NC; ++a)
        for (int b = 0; b < NC; ++b) {
            out[2 * (base + a * NC + b)] = (D)(double)in[2 * (base + b * NC + a)];
            out[2 * (base + a * NC + b) + 1] = (D)(-(double)in[2 * (base + b * NC + a) + 1]);
        }
}

int launch_stout_backward(const void *U, const void *G_V, void *G_U, const Lat &g, int nc, dirac_prec prec, double rho,
                          int nsteps, cudaStream_t s) {
    const size_t field = (size_t)g.V * 4 * nc * nc * 2;   // scalars per field
    const size_t eb = elem_bytes(prec);
    void *steps = nullptr;   // U^(1) .. U^(nsteps-1) in the storage precision
    double *sa = nullptr, *sb = nullptr, *y = nullptr;
    int rc = DIRAC_OK;
    auto fail = [&](int r) {
        cudaStreamSynchronize(s);
        cudaFree(steps);
        cudaFree(sa);
        cudaFree(sb);
        cudaFree(y);
        return r;
    };
    if (nsteps > 1 && cudaMalloc(&steps, (size_t)(nsteps - 1) * field * eb) != cudaSuccess) return fail(DIRAC_ERR_OOM);
    if (cudaMalloc(&sa, field * 8) != cudaSuccess || cudaMalloc(&sb, field * 8) != cudaSuccess ||
        cudaMalloc(&y, field * 8) != cudaSuccess) {
        cudaGetLastError();
        return fail(DIRAC_ERR_OOM);
    }
    auto field_ptr = [&](int i) -> const void * {
        return i == 0 ? U : (const void *)((const char *)steps + (size_t)(i - 1) * field * eb);
    };
    rc = dispatch_uprec(prec, [&](auto utag) {
        using UE = std::remove_pointer_t<decltype(utag)>;
        // N_c 1..4: the 2N_c x 2N_c block exponential stays small in registers
        return dispatch_nc<false>(nc, [&](auto ncc) {
            constexpr int NC = decltype(ncc)::value;
            const long long links = g.V * 4;
            // forward: the inputs of every step (U^(0) = U)
            for (int i = 1; i < nsteps; ++i) {
                stout_step_kernel<NC, UE><<<grid_for(links, 128), 128, 0, s>>>((const UE *)field_ptr(i - 1),
                                                                                (UE *)field_ptr(i), g, rho);
                const int e = launch_check("stout_step_kernel");
                if (e) return e;
            }
            // Sigma = G_V^dag in FP64, then back through the steps
            dagger_links_kernel<NC, UE, double><<<grid_for(links, 128), 128, 0, s>>>((const UE *)G_V, sa, links);
            double *cur = sa, *nxt = sb;
            for (int i = nsteps - 1; i >= 0; --i) {
                stout_back_own_kernel<NC, UE><<<grid_for(links, 128), 128, 0, s>>>((const UE *)field_ptr(i), cur, nxt,
                                                                                    y, g, rho);
                stout_back_staple_kernel<NC, UE><<<grid_for(links, 128), 128, 0, s>>>((const UE *)field_ptr(i), y, nxt,
                                                                                       g, rho);
                const int e = launch_check("stout backward");
                if (e) return e;
                double *t = cur;
                cur = nxt;
                nxt = t;
            }
            dagger_links_kernel<NC, double, UE><<<grid_for(links, 128), 128, 0, s>>>(cur, (UE *)G_U, links);
            return launch_check("dagger_links_kernel");
        });
    });
    if (!rc) rc = cuda_check(cudaStreamSynchronize(s), "stout backward sync");
    return fail(rc);
}

int launch_stout_step(const void *U, void *out, const Lat &g, int nc, dirac_prec prec, double rho, cudaStream_t s) {
    return dispatch_uprec(prec, [&](auto utag) {
        using UE = std::remove_pointer_t<decltype(utag)>;
        return dispatch_nc(nc, [&](auto ncc) {
            constexpr int NC = decltype(ncc)::value;
            const long long threads = g.V * 4;
            stout_step_kernel<NC, UE><<<grid_for(threads, 128), 128, 0, s>>>((const UE *)U, (UE *)out, g, rho);
            return launch_check("stout_step_kernel");
        });
    });
}

}  // namespace dgb
