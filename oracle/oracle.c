/*
 * oracle.c -- plain, slow, FP64 CPU reference for the multi-RHS Dirac operators
 * of Duerr, "Fast and flexible implementations of Wilson, Brillouin and Susskind
 * fermions in lattice QCD" (arXiv:2112.14640).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library calls this file; only the
 * tests, the smoke check and the CPU-baseline leg of the benchmark load it.
 * It shares no code, header, table or helper with the CUDA path.
 *
 * Every routine writes out the paper's definition literally:
 *   - full 4x4 gamma matrices (chiral representation, App. A) instead of the
 *     spin-projection trick,
 *   - W links by explicit enumeration of all k! minimal hop orderings
 *     (Tab. "off-axis"), all 80 off-centre directions stored,
 *   - periodic index arithmetic with boundary phases folded into a copy of
 *     the links (one multiplication of U_mu(n) by bc[mu] where n_mu = N_mu-1).
 * OpenMP only distributes independent output sites; no blocking or fusion.
 *
 * Layouts (all complex double, C order, x fastest among the coordinates):
 *   site n  = ((t*Nz + z)*Ny + y)*Nx + x
 *   U[n][mu][a][b]             mu = 0..3 <-> x,y,z,t (paper's mu = 1..4)
 *   W[n][dir][a][b]            dir = (st+1)*27+(sz+1)*9+(sy+1)*3+(sx+1), 0..80,
 *                              dir 40 is the centre (identity)
 *   Wilson-type psi[n][c][s][v]   staggered phi[n][c][v]   (v = RHS index)
 *
 * Parity status: every function here is pinned by the CPU tests
 * (free-field symbols, gamma5-hermiticity, gauge covariance, W identities,
 * dense brute force, solver residuals, finite differences for the force,
 * the abelian closed form and pure-gauge zero of the field strength).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ---------------------------------------------------------------- geometry */

static long vol4(const int d[4]) { return (long)d[0] * d[1] * d[2] * d[3]; }

static void coords(const int d[4], long n, int x[4]) {
    x[0] = (int)(n % d[0]); n /= d[0];
    x[1] = (int)(n % d[1]); n /= d[1];
    x[2] = (int)(n % d[2]); n /= d[2];
    x[3] = (int)n;
}

static long index_of(const int d[4], const int x[4]) {
    int y[4];
    for (int m = 0; m < 4; ++m) y[m] = ((x[m] % d[m]) + d[m]) % d[m];  /* periodic */
    return (((long)y[3] * d[2] + y[2]) * d[1] + y[1]) * d[0] + y[0];
}

static long shifted(const int d[4], long n, const int s[4]) {
    int x[4];
    coords(d, n, x);
    for (int m = 0; m < 4; ++m) x[m] += s[m];
    return index_of(d, x);
}

static long hop(const int d[4], long n, int mu, int sign) {
    int s[4] = {0, 0, 0, 0};
    s[mu] = sign;
    return shifted(d, n, s);
}

/* ------------------------------------------------------- gamma matrices (App. A)
 * Chiral (Weyl) representation, gamma_1..gamma_4 <-> x,y,z,t; gamma_5 = diag(1,1,-1,-1). */

static void gamma_matrix(int mu, cplx g[4][4]) {
    memset(g, 0, sizeof(cplx) * 16);
    const cplx im = _Complex_I;
    switch (mu) {
    case 0: g[0][3] = -im; g[1][2] = -im; g[2][1] = im; g[3][0] = im; break;
    case 1: g[0][3] = -1; g[1][2] = 1;  g[2][1] = 1;  g[3][0] = -1; break;
    case 2: g[0][2] = -im; g[1][3] = im; g[2][0] = im; g[3][1] = -im;break;
    case 3: g[0][2] = 1;  g[1][3] = 1;  g[2][0] = 1;  g[3][1] = 1;  break;
    }
}

void orc_gamma(int mu, double *out /* 4x4 complex, row-major */) {
    cplx g[4][4];
    gamma_matrix(mu, g);
    memcpy(out, g, sizeof(g));
}

/* --------------------------------------------------------- colour algebra */

static void mat_mul(int nc, const cplx *A, const cplx *B, cplx *C) {
    for (int a = 0; a < nc; ++a)
        for (int b = 0; b < nc; ++b) {
            cplx acc = 0;
            for (int k = 0; k < nc; ++k) acc += A[a * nc + k] * B[k * nc + b];
            C[a * nc + b] = acc;
        }
}

static void mat_dag(int nc, const cplx *A, cplx *B) {
    for (int a = 0; a < nc; ++a)
        for (int b = 0; b < nc; ++b) B[a * nc + b] = conj(A[b * nc + a]);
}

/* ------------------------------------------------------- boundary phases
 * Reading of the boundary conditions: U_mu(n) -> bc[mu] * U_mu(n) on the links
 * with n_mu = N_mu - 1 (the links that wrap around); everything else periodic. */

void orc_phase_links(const int d[4], int nc, const int bc[4], const cplx *U, cplx *Up) {
    const long V = vol4(d);
    const long per = (long)nc * nc;
#pragma omp parallel for
    for (long n = 0; n < V; ++n) {
        int x[4];
        coords(d, n, x);
        for (int mu = 0; mu < 4; ++mu) {
            double ph = (x[mu] == d[mu] - 1) ? (double)bc[mu] : 1.0;
            const cplx *src = U + (n * 4 + mu) * per;
            cplx *dst = Up + (n * 4 + mu) * per;
            for (long e = 0; e < per; ++e) dst[e] = ph * src[e];
        }
    }
}

/* link V_{sign*mu}(n): V_mu(n) for sign=+1, V_mu(n-mu)^dagger for sign=-1 */
static void signed_link(const int d[4], int nc, const cplx *U, long n, int mu, int sign, cplx *out) {
    const long per = (long)nc * nc;
    if (sign > 0) {
        memcpy(out, U + (n * 4 + mu) * per, sizeof(cplx) * per);
    } else {
        long m = hop(d, n, mu, -1);
        mat_dag(nc, U + (m * 4 + mu) * per, out);
    }
}

/* ------------------------------------------------ Wilson Dirac operator
 * Eq. (app_wils), r = 1, c_SW = 0:
 *   (D_W psi)(n) = 1/2 sum_mu { [(gamma_mu - 1) (x) U_mu(n)] psi(n+mu)
 *                             - [(gamma_mu + 1) (x) U_mu(n-mu)^dag] psi(n-mu) }
 *                  + (4 + m0) psi(n)
 * U must already carry the boundary phases (orc_phase_links). */

static void wilson_site(const int d[4], int nc, int nv, const cplx *U, double m0,
                        const cplx *in, long n, cplx *o) {
    const long per_site = (long)nc * 4 * nv;
    cplx g[4][4][4];
    for (int mu = 0; mu < 4; ++mu) gamma_matrix(mu, g[mu]);
    {
        const cplx *c0 = in + n * per_site;
        for (long e = 0; e < per_site; ++e) o[e] = (4.0 + m0) * c0[e];
        cplx L[64];
        for (int mu = 0; mu < 4; ++mu)
            for (int sign = 1; sign >= -1; sign -= 2) {
                long m = hop(d, n, mu, sign);
                signed_link(d, nc, U, n, mu, sign, L);
                /* spin matrix: +1/2 (gamma - 1) forward, -1/2 (gamma + 1) backward */
                cplx S[4][4];
                for (int a = 0; a < 4; ++a)
                    for (int b = 0; b < 4; ++b) {
                        cplx id = (a == b) ? 1.0 : 0.0;
                        S[a][b] = (sign > 0) ? 0.5 * (g[mu][a][b] - id) : -0.5 * (g[mu][a][b] + id);
                    }
                const cplx *pm = in + m * per_site;
                for (int c = 0; c < nc; ++c)
                    for (int s = 0; s < 4; ++s)
                        for (int v = 0; v < nv; ++v) {
                            cplx acc = 0;
                            for (int c2 = 0; c2 < nc; ++c2)
                                for (int s2 = 0; s2 < 4; ++s2)
                                    acc += S[s][s2] * L[c * nc + c2] * pm[((long)c2 * 4 + s2) * nv + v];
                            o[((long)c * 4 + s) * nv + v] += acc;
                        }
            }
    }
}

void orc_wilson(const int d[4], int nc, int nv, const cplx *U, double m0,
                const cplx *in, cplx *out) {
    const long V = vol4(d);
#pragma omp parallel for
    for (long n = 0; n < V; ++n) wilson_site(d, nc, nv, U, m0, in, n, out + n * (long)nc * 4 * nv);
}

/* output only at the listed sites: out[i] = (D psi)(sites[i]) */
void orc_wilson_sites(const int d[4], int nc, int nv, const cplx *U, double m0,
                      const cplx *in, const long *sites, long ns, cplx *out) {
#pragma omp parallel for
    for (long i = 0; i < ns; ++i) wilson_site(d, nc, nv, U, m0, in, sites[i], out + i * (long)nc * 4 * nv);
}

/* ------------------------------------------------ staggered Dirac operator
 * Eq. (def_stag):
 *   (D_S phi)(n) = sum_mu eta_mu(n) 1/2 [U_mu(n) phi(n+mu) - U_mu(n-mu)^dag phi(n-mu)] + m0 phi(n)
 * eta_1 = 1, eta_2 = (-1)^x, eta_3 = (-1)^(x+y), eta_4 = (-1)^(x+y+z) with the
 * paper's 1-based coordinates (App. D toggles eta_2 to -1 at x = 1); with
 * 0-based x here the exponent is sum_{nu<mu} (x_nu + 1). */

static double eta(const int x[4], int mu) {
    int e = 0;
    for (int nu = 0; nu < mu; ++nu) e += x[nu] + 1;
    return (e & 1) ? -1.0 : 1.0;
}

static void staggered_site(const int d[4], int nc, int nv, const cplx *U, double m0,
                           const cplx *in, long n, cplx *o) {
    const long per_site = (long)nc * nv;
    {
        int x[4];
        coords(d, n, x);
        const cplx *c0 = in + n * per_site;
        for (long e = 0; e < per_site; ++e) o[e] = m0 * c0[e];
        cplx L[64];
        for (int mu = 0; mu < 4; ++mu)
            for (int sign = 1; sign >= -1; sign -= 2) {
                long m = hop(d, n, mu, sign);
                signed_link(d, nc, U, n, mu, sign, L);
                double f = 0.5 * sign * eta(x, mu);
                const cplx *pm = in + m * per_site;
                for (int c = 0; c < nc; ++c)
                    for (int v = 0; v < nv; ++v) {
                        cplx acc = 0;
                        for (int c2 = 0; c2 < nc; ++c2) acc += L[c * nc + c2] * pm[(long)c2 * nv + v];
                        o[(long)c * nv + v] += f * acc;
                    }
            }
    }
}

void orc_staggered(const int d[4], int nc, int nv, const cplx *U, double m0,
                   const cplx *in, cplx *out) {
    const long V = vol4(d);
#pragma omp parallel for
    for (long n = 0; n < V; ++n) staggered_site(d, nc, nv, U, m0, in, n, out + n * (long)nc * nv);
}

void orc_staggered_sites(const int d[4], int nc, int nv, const cplx *U, double m0,
                         const cplx *in, const long *sites, long ns, cplx *out) {
#pragma omp parallel for
    for (long i = 0; i < ns; ++i) staggered_site(d, nc, nv, U, m0, in, sites[i], out + i * (long)nc * nv);
}

/* -------------------------------------------------- W links (Tab. off-axis)
 * W_s(n) = (1/k!) sum over the k! orderings of the k hops of the product of
 * signed links along the path from n to n+s; s in {-1,0,1}^4, k = |s|_1.
 * All 80 off-centre directions are enumerated directly (no W_{-s}(n) =
 * W_s(n-s)^dag shortcut); dir 40 is set to the identity. */

static int next_perm(int *a, int k) {       /* lexicographic successor */
    int i = k - 2;
    while (i >= 0 && a[i] >= a[i + 1]) --i;
    if (i < 0) return 0;
    int j = k - 1;
    while (a[j] <= a[i]) --j;
    int t = a[i]; a[i] = a[j]; a[j] = t;
    for (int l = i + 1, r = k - 1; l < r; ++l, --r) { t = a[l]; a[l] = a[r]; a[r] = t; }
    return 1;
}

void orc_dir_offset(int dir, int s[4]) {
    s[0] = dir % 3 - 1;
    s[1] = (dir / 3) % 3 - 1;
    s[2] = (dir / 9) % 3 - 1;
    s[3] = (dir / 27) % 3 - 1;
}

/* the 81 W_s(n) of one site into Wn[81][nc][nc] */
static void build_w_site(const int d[4], int nc, const cplx *U, long n, cplx *Wn) {
    const long per = (long)nc * nc;
    {
        cplx P[64], T[64], L[64];
        for (int dir = 0; dir < 81; ++dir) {
            cplx *w = Wn + dir * per;
            int s[4];
            orc_dir_offset(dir, s);
            int axes[4], k = 0;
            for (int m = 0; m < 4; ++m)
                if (s[m] != 0) axes[k++] = m;
            memset(w, 0, sizeof(cplx) * per);
            if (k == 0) {
                for (int a = 0; a < nc; ++a) w[a * nc + a] = 1.0;
                continue;
            }
            int perm[4];
            for (int i = 0; i < k; ++i) perm[i] = axes[i];
            int npaths = 0;
            do {
                for (long e = 0; e < per; ++e) P[e] = 0;
                for (int a = 0; a < nc; ++a) P[a * nc + a] = 1.0;
                long pos = n;
                for (int i = 0; i < k; ++i) {
                    int mu = perm[i];
                    signed_link(d, nc, U, pos, mu, s[mu], L);
                    mat_mul(nc, P, L, T);
                    memcpy(P, T, sizeof(cplx) * per);
                    pos = hop(d, pos, mu, s[mu]);
                }
                for (long e = 0; e < per; ++e) w[e] += P[e];
                ++npaths;
            } while (next_perm(perm, k));
            for (long e = 0; e < per; ++e) w[e] /= (double)npaths;
        }
    }
}

void orc_build_w(const int d[4], int nc, const cplx *U, cplx *W) {
    const long V = vol4(d);
#pragma omp parallel for
    for (long n = 0; n < V; ++n) build_w_site(d, nc, U, n, W + n * 81 * (long)nc * nc);
}

void orc_build_w_sites(const int d[4], int nc, const cplx *U, const long *sites, long ns, cplx *W) {
#pragma omp parallel for
    for (long i = 0; i < ns; ++i) build_w_site(d, nc, U, sites[i], W + i * 81 * (long)nc * nc);
}

/* ------------------------------------------------ Brillouin Dirac operator
 * Eq. (app_bril) with Eqs. (def_ider, def_blap), r = 1, c_SW = 0:
 *   (D_B psi)(n) = (m0 - lambda_0/2) psi(n)
 *      + sum_{s != 0} [ rho_k sum_mu s_mu gamma_mu - lambda_k/2 ] (x) W_s(n) psi(n+s)
 * with rho = (64,16,4,1)/432, lambda = (-240,8,4,2,1)/64, k = |s|_1.
 * Reading: the derivative carries sum_mu s_mu gamma_mu (every axis the offset
 * moves along), as Eq. (def_ider) implies. */

static const double RHO[5] = {0.0, 64.0 / 432.0, 16.0 / 432.0, 4.0 / 432.0, 1.0 / 432.0};
static const double LAM[5] = {-240.0 / 64.0, 8.0 / 64.0, 4.0 / 64.0, 2.0 / 64.0, 1.0 / 64.0};

/* one output site n; Wn = the 81 W_s(n) of that site */
static void brillouin_site(const int d[4], int nc, int nv, const cplx *Wn, double m0,
                           const cplx *in, long n, cplx *o) {
    const long per_site = (long)nc * 4 * nv;
    const long per = (long)nc * nc;
    cplx g[4][4][4];
    for (int mu = 0; mu < 4; ++mu) gamma_matrix(mu, g[mu]);
    {
        for (long e = 0; e < per_site; ++e) o[e] = 0;
        for (int dir = 0; dir < 81; ++dir) {
            int s[4];
            orc_dir_offset(dir, s);
            int k = abs(s[0]) + abs(s[1]) + abs(s[2]) + abs(s[3]);
            cplx S[4][4];
            for (int a = 0; a < 4; ++a)
                for (int b = 0; b < 4; ++b) {
                    cplx v = 0;
                    for (int mu = 0; mu < 4; ++mu) v += RHO[k] * s[mu] * g[mu][a][b];
                    if (a == b) v += (k == 0) ? (m0 - 0.5 * LAM[0]) : -0.5 * LAM[k];
                    S[a][b] = v;
                }
            long m = shifted(d, n, s);
            const cplx *w = Wn + dir * per;
            const cplx *pm = in + m * per_site;
            for (int c = 0; c < nc; ++c)
                for (int sp = 0; sp < 4; ++sp)
                    for (int v = 0; v < nv; ++v) {
                        cplx acc = 0;
                        for (int c2 = 0; c2 < nc; ++c2)
                            for (int s2 = 0; s2 < 4; ++s2)
                                acc += S[sp][s2] * w[c * nc + c2] * pm[((long)c2 * 4 + s2) * nv + v];
                        o[((long)c * 4 + sp) * nv + v] += acc;
                    }
        }
    }
}

void orc_brillouin(const int d[4], int nc, int nv, const cplx *W, double m0,
                   const cplx *in, cplx *out) {
    const long V = vol4(d);
    const long per_site = (long)nc * 4 * nv;
#pragma omp parallel for
    for (long n = 0; n < V; ++n) brillouin_site(d, nc, nv, W + n * 81 * (long)nc * nc, m0, in, n, out + n * per_site);
}

/* sampled sites: Wsites[i] holds the 81 W of sites[i] (orc_build_w_sites) */
void orc_brillouin_sites(const int d[4], int nc, int nv, const cplx *Wsites, double m0,
                         const cplx *in, const long *sites, long ns, cplx *out) {
    const long per_site = (long)nc * 4 * nv;
#pragma omp parallel for
    for (long i = 0; i < ns; ++i)
        brillouin_site(d, nc, nv, Wsites + i * 81 * (long)nc * nc, m0, in, sites[i], out + i * per_site);
}

/* ------------------------------------------------- Laplace operators (Sec. 6, 7)
 * The "embedded" Laplace operators A = -1/2 Lap + m^2/2, acting trivially in
 * spin: on ns = 4 spin components per colour (Wilson-type vectors, the
 * paper's wlap/blap) or ns = 1 (colour-only vectors, wsuv/bsuv, App. F).
 *   Eq. (app_wlap): (A psi)(n) = (4 + m^2/2) psi(n)
 *        - 1/2 sum_mu [ U_mu(n) psi(n+mu) + U_mu(n-mu)^dag psi(n-mu) ]
 *   Eq. (app_blap): (A psi)(n) = (m^2/2 - lambda_0/2) psi(n)
 *        - 1/2 sum_{s != 0} lambda_k W_s(n) psi(n+s)
 * Vectors are [site][colour][spin][v] (ns = 4) or [site][colour][v] (ns = 1). */

static void wlap_site(const int d[4], int nc, int ns, int nv, const cplx *U, double m,
                      const cplx *in, long n, cplx *o) {
    const long per_site = (long)nc * ns * nv;
    const cplx *c0 = in + n * per_site;
    for (long e = 0; e < per_site; ++e) o[e] = (4.0 + 0.5 * m * m) * c0[e];
    cplx L[64];
    for (int mu = 0; mu < 4; ++mu)
        for (int sign = 1; sign >= -1; sign -= 2) {
            long nb = hop(d, n, mu, sign);
            signed_link(d, nc, U, n, mu, sign, L);
            const cplx *pm = in + nb * per_site;
            for (int c = 0; c < nc; ++c)
                for (int sp = 0; sp < ns; ++sp)
                    for (int v = 0; v < nv; ++v) {
                        cplx acc = 0;
                        for (int c2 = 0; c2 < nc; ++c2) acc += L[c * nc + c2] * pm[((long)c2 * ns + sp) * nv + v];
                        o[((long)c * ns + sp) * nv + v] -= 0.5 * acc;
                    }
        }
}

void orc_wlap(const int d[4], int nc, int ns, int nv, const cplx *U, double m, const cplx *in, cplx *out) {
    const long V = vol4(d);
#pragma omp parallel for
    for (long n = 0; n < V; ++n) wlap_site(d, nc, ns, nv, U, m, in, n, out + n * (long)nc * ns * nv);
}

void orc_wlap_sites(const int d[4], int nc, int ns, int nv, const cplx *U, double m, const cplx *in,
                    const long *sites, long nsites, cplx *out) {
#pragma omp parallel for
    for (long i = 0; i < nsites; ++i) wlap_site(d, nc, ns, nv, U, m, in, sites[i], out + i * (long)nc * ns * nv);
}

/* one output site n; Wn = the 81 W_s(n) of that site (centre = identity) */
static void blap_site(const int d[4], int nc, int ns, int nv, const cplx *Wn, double m,
                      const cplx *in, long n, cplx *o) {
    const long per_site = (long)nc * ns * nv;
    const long per = (long)nc * nc;
    for (long e = 0; e < per_site; ++e) o[e] = 0;
    for (int dir = 0; dir < 81; ++dir) {
        int s[4];
        orc_dir_offset(dir, s);
        int k = abs(s[0]) + abs(s[1]) + abs(s[2]) + abs(s[3]);
        double f = (k == 0) ? 0.5 * m * m - 0.5 * LAM[0] : -0.5 * LAM[k];
        long nb = shifted(d, n, s);
        const cplx *w = Wn + dir * per;
        const cplx *pm = in + nb * per_site;
        for (int c = 0; c < nc; ++c)
            for (int sp = 0; sp < ns; ++sp)
                for (int v = 0; v < nv; ++v) {
                    cplx acc = 0;
                    for (int c2 = 0; c2 < nc; ++c2) acc += w[c * nc + c2] * pm[((long)c2 * ns + sp) * nv + v];
                    o[((long)c * ns + sp) * nv + v] += f * acc;
                }
    }
}

void orc_blap(const int d[4], int nc, int ns, int nv, const cplx *W, double m, const cplx *in, cplx *out) {
    const long V = vol4(d);
    const long per_site = (long)nc * ns * nv;
#pragma omp parallel for
    for (long n = 0; n < V; ++n) blap_site(d, nc, ns, nv, W + n * 81 * (long)nc * nc, m, in, n, out + n * per_site);
}

void orc_blap_sites(const int d[4], int nc, int ns, int nv, const cplx *Wsites, double m, const cplx *in,
                    const long *sites, long nsites, cplx *out) {
    const long per_site = (long)nc * ns * nv;
#pragma omp parallel for
    for (long i = 0; i < nsites; ++i)
        blap_site(d, nc, ns, nv, Wsites + i * 81 * (long)nc * nc, m, in, sites[i], out + i * per_site);
}

/* ------------------------------------- clover-leaf field strength (Sec. 5)
 * Eq. (def_clov) needs the hermitian "clover-leaf" field strength F_mu,nu(n)
 * but the paper does not write it out.  Reading: Q_mu,nu(n) is the sum of the
 * four plaquettes of the (mu,nu) plane that have n as a corner, each one a
 * closed path from n back to n turning the same way (a step along the first
 * direction, then along the second), and
 *   F_mu,nu(n) = (Q_mu,nu(n) - Q_mu,nu(n)^dag) / (8 i),
 * with no trace subtracted.  The six orientations are stored in the paper's
 * order (mu,nu) = (1,2),(1,3),(1,4),(2,3),(2,4),(3,4), i.e. 0-based
 * (0,1),(0,2),(0,3),(1,2),(1,3),(2,3):  F[n][6][a][b].
 * Closed loops do not see the boundary phases, so U may carry them or not. */

/* product along the closed path n -> n+a -> n+a+b -> n+b -> n, where a and b
 * are signed unit steps (direction, sign): V_a(n) V_b(n+a) V_-a(n+a+b) V_-b(n+b) */
static void leaf(const int d[4], int nc, const cplx *U, long n, int amu, int as, int bmu, int bs, cplx *out) {
    const long per = (long)nc * nc;
    cplx *L = malloc(sizeof(cplx) * per), *T = malloc(sizeof(cplx) * per);
    int sa[4] = {0, 0, 0, 0}, sb[4] = {0, 0, 0, 0}, sab[4] = {0, 0, 0, 0};
    sa[amu] = as;
    sb[bmu] = bs;
    sab[amu] += as;
    sab[bmu] += bs;
    const long na = shifted(d, n, sa), nb = shifted(d, n, sb), nab = shifted(d, n, sab);
    signed_link(d, nc, U, n, amu, as, out);
    signed_link(d, nc, U, na, bmu, bs, L);
    mat_mul(nc, out, L, T);
    signed_link(d, nc, U, nab, amu, -as, L);
    mat_mul(nc, T, L, out);
    signed_link(d, nc, U, nb, bmu, -bs, L);
    mat_mul(nc, out, L, T);
    memcpy(out, T, sizeof(cplx) * per);
    free(L);
    free(T);
}

void orc_field_strength(const int d[4], int nc, const cplx *U, cplx *F) {
    const long V = vol4(d);
    const long per = (long)nc * nc;
#pragma omp parallel for
    for (long n = 0; n < V; ++n) {
        cplx *Q = malloc(sizeof(cplx) * per), *P = malloc(sizeof(cplx) * per);
        int k = 0;
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = mu + 1; nu < 4; ++nu, ++k) {
                memset(Q, 0, sizeof(cplx) * per);
                /* the four leaves: (+mu,+nu), (+nu,-mu), (-mu,-nu), (-nu,+mu) */
                const int steps[4][4] = {{mu, 1, nu, 1}, {nu, 1, mu, -1}, {mu, -1, nu, -1}, {nu, -1, mu, 1}};
                for (int l = 0; l < 4; ++l) {
                    leaf(d, nc, U, n, steps[l][0], steps[l][1], steps[l][2], steps[l][3], P);
                    for (long e = 0; e < per; ++e) Q[e] += P[e];
                }
                cplx *f = F + (n * 6 + k) * per;
                for (int a = 0; a < nc; ++a)
                    for (int b = 0; b < nc; ++b)
                        f[a * nc + b] = (Q[a * nc + b] - conj(Q[b * nc + a])) / (8.0 * _Complex_I);
            }
        free(Q);
        free(P);
    }
}

/* ------------------------------------------ gamma_5 and epsilon (Sec. 3)
 * gamma_5 = diag(1,1,-1,-1) in spinor space; epsilon(n) = (-1)^(x+y+z+t). */

void orc_gamma5(const int d[4], int nc, int nv, const cplx *in, cplx *out) {
    const long V = vol4(d);
#pragma omp parallel for
    for (long n = 0; n < V; ++n)
        for (int c = 0; c < nc; ++c)
            for (int s = 0; s < 4; ++s)
                for (int v = 0; v < nv; ++v) {
                    long i = ((n * nc + c) * 4 + s) * nv + v;
                    out[i] = (s < 2) ? in[i] : -in[i];
                }
}

void orc_epsilon(const int d[4], int nc, int nv, const cplx *in, cplx *out) {
    const long V = vol4(d);
#pragma omp parallel for
    for (long n = 0; n < V; ++n) {
        int x[4];
        coords(d, n, x);
        double e = ((x[0] + x[1] + x[2] + x[3]) & 1) ? -1.0 : 1.0;
        for (long i = 0; i < (long)nc * nv; ++i) out[n * nc * nv + i] = e * in[n * nc * nv + i];
    }
}
