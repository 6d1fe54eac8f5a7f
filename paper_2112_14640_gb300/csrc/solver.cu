// solver.cu -- Krylov solvers of Sec. 9 on the multi-RHS operators:
//  * CG on the normal equations D^dag D x = D^dag b (one independent
//    recursion per RHS: own alpha^(i), beta^(i));
//  * BiCGstab on D x = b (van der Vorst, shadow residual r_hat = r_0);
//  * defect correction ("mixed precision" solvers of Sec. 9): the residual
//    r = b - A x, its norm, the convergence test and the update x += e are
//    done in the operator's precision, the correction e comes from a Krylov
//    solve of A e = r/|r| in a lower storage precision (BF16/FP16/FP32
//    links and vectors, FP32 arithmetic, FP64 reductions).
// Recompute/exit rules (Sec. 9): recompute r = b - A x when the iteration
// count is a multiple of recompute_every, when every active RHS's updated
// residual passes, or at maxit; exit when all recomputed residuals pass, when
// updated and recomputed norms of an unconverged RHS differ by more than 1%,
// or at maxit.  An RHS whose recomputed residual passes is frozen
// (alpha = beta = 0) while the others continue.
//
// Per-RHS coefficients are formed on the device from FP64 reductions; the
// host reads the N_v residual norms once per iteration to apply the rules.
#include <math.h>
#include <string.h>

#include <chrono>
#include <vector>

#include "internal.h"

namespace dgb {

constexpr int kWsVecs = 8;
constexpr int kNS = 64;   // max RHS

struct Ws {
    void *v[kWsVecs];
    double *rr, *rr_new, *pq, *alpha, *beta, *act, *nb, *c1, *c2, *c3, *omega, *rho, *rho_new, *tt;
};

static int get_ws(const dirac_op *op, Ws &w) {
    dirac_op *self = (dirac_op *)op;
    const size_t scal = 16 * kNS * 2 * sizeof(double);
    const size_t need = kWsVecs * op->vec_bytes + scal;
    if (!self->solver_ws) {
        if (cudaMalloc(&self->solver_ws, need) != cudaSuccess) {
            cudaGetLastError();
            self->solver_ws = nullptr;
            return DIRAC_ERR_OOM;
        }
        self->solver_ws_bytes = need;
    }
    char *base = (char *)self->solver_ws;
    for (int i = 0; i < kWsVecs; ++i) w.v[i] = base + i * op->vec_bytes;
    double *d = (double *)(base + kWsVecs * op->vec_bytes);
    double **arr[] = {&w.rr, &w.rr_new, &w.pq, &w.alpha, &w.beta, &w.act, &w.nb, &w.c1,
                      &w.c2, &w.c3, &w.omega, &w.rho, &w.rho_new, &w.tt};
    for (size_t i = 0; i < sizeof(arr) / sizeof(arr[0]); ++i) *arr[i] = d + i * kNS * 2;
    return DIRAC_OK;
}

// The operator's solver workspace: the first nvecs vectors and the scalar
// area (arrays of 2*64 doubles in the order rr, rr_new, pq, alpha, beta, act,
// nb, ...), for drivers in other translation units.
static int apply_A_pq(const dirac_op *op, const void *p, void *q, double *pq, double m0, cudaStream_t s);

int batch_apply_A_pq(const dirac_op *op, const void *p, void *q, double *pq, double m0, cudaStream_t s) {
    return apply_A_pq(op, p, q, pq, m0, s);
}

int solver_ws(const dirac_op *op, void **vecs, int nvecs, double **scal) {
    Ws w;
    int rc = get_ws(op, w);
    if (rc) return rc;
    for (int i = 0; i < nvecs && i < kWsVecs; ++i) vecs[i] = w.v[i];
    *scal = w.rr;
    return DIRAC_OK;
}

// ---------------------------------------------------------------- coefficient kernels
// alpha = rr / <p, A p>; pq holds N_v real values <p, D^dag D p> = |D p|^2
__global__ void cg_alpha_kernel(int nv, const double *rr, const double *pq, const double *act, double *alpha) {
    const int v = threadIdx.x;
    if (v >= nv) return;
    const double p = pq[v];
    const double a = (act[v] != 0.0 && p != 0.0) ? rr[v] / p : 0.0;
    alpha[2 * v] = a;
    alpha[2 * v + 1] = 0.0;
}

__global__ void cg_beta_kernel(int nv, const double *rr_new, double *rr, const double *act, double *beta) {
    const int v = threadIdx.x;
    if (v >= nv) return;
    const double b = (act[v] != 0.0 && rr[v] != 0.0) ? rr_new[v] / rr[v] : 0.0;
    beta[2 * v] = b;
    beta[2 * v + 1] = 0.0;
    rr[v] = rr_new[v];
}

__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    const double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double2 cmuld(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// beta = (rho_new/rho) (alpha/omega); c1 = beta, c2 = -beta*omega; flags breakdown in act (=0)
__global__ void bicg_beta_kernel(int nv, const double *rho_new, const double *rho, const double *alpha,
                                 const double *omega, double *act, double *beta, double *c2, double *brk) {
    const int v = threadIdx.x;
    if (v >= nv) return;
    double2 rn = make_double2(rho_new[2 * v], rho_new[2 * v + 1]);
    double2 ro = make_double2(rho[2 * v], rho[2 * v + 1]);
    double2 al = make_double2(alpha[2 * v], alpha[2 * v + 1]);
    double2 om = make_double2(omega[2 * v], omega[2 * v + 1]);
    double2 b = make_double2(0, 0);
    if (act[v] != 0.0) {
        if (hypot(rn.x, rn.y) == 0.0 || hypot(om.x, om.y) == 0.0) {
            act[v] = 0.0;
            brk[v] = 1.0;
        } else {
            b = cmuld(cdiv(rn, ro), cdiv(al, om));
        }
    }
    beta[2 * v] = b.x;
    beta[2 * v + 1] = b.y;
    double2 bo = cmuld(b, om);
    c2[2 * v] = -bo.x;
    c2[2 * v + 1] = -bo.y;
}

// alpha = rho_new / <rhat, v>
__global__ void bicg_alpha_kernel(int nv, const double *rho_new, const double *rv, const double *act, double *alpha) {
    const int v = threadIdx.x;
    if (v >= nv) return;
    double2 a = make_double2(0, 0);
    double2 d = make_double2(rv[2 * v], rv[2 * v + 1]);
    if (act[v] != 0.0 && (d.x != 0.0 || d.y != 0.0))
        a = cdiv(make_double2(rho_new[2 * v], rho_new[2 * v + 1]), d);
    alpha[2 * v] = a.x;
    alpha[2 * v + 1] = a.y;
}

// omega = <t, s> / <t, t>; rho = rho_new
__global__ void bicg_omega_kernel(int nv, const double *ts, const double *tt, const double *act, double *omega,
                                  const double *rho_new, double *rho, double *brk, double *actw) {
    const int v = threadIdx.x;
    if (v >= nv) return;
    double2 o = make_double2(0, 0);
    if (act[v] != 0.0 && tt[v] > 0.0) o = make_double2(ts[2 * v] / tt[v], ts[2 * v + 1] / tt[v]);
    if (act[v] != 0.0 && o.x == 0.0 && o.y == 0.0) {
        brk[v] = 1.0;
        actw[v] = 0.0;
    }
    omega[2 * v] = o.x;
    omega[2 * v + 1] = o.y;
    rho[2 * v] = rho_new[2 * v];
    rho[2 * v + 1] = rho_new[2 * v + 1];
}

// c[2v] = act ? f(|x|) : 0 with f(r) = scale / r (inverse) or r / scale
__global__ void coef_from_norm_kernel(int nv, const double *rr, const double *act, double *c, int inverse,
                                      double scale = 1.0) {
    const int v = threadIdx.x;
    if (v >= nv) return;
    double r = sqrt(rr[v]);
    double val = (act[v] != 0.0 && r > 0.0) ? (inverse ? scale / r : r / scale) : 0.0;
    c[2 * v] = val;
    c[2 * v + 1] = 0.0;
}

// ---------------------------------------------------------------- host helpers
static int to_host(double *h, const double *d, int n, cudaStream_t s) {
    int rc = cuda_check(cudaMemcpyAsync(h, d, n * sizeof(double), cudaMemcpyDeviceToHost, s), "D2H scalars");
    if (!rc) rc = cuda_check(cudaStreamSynchronize(s), "solver sync");
    return rc;
}
static int to_dev(double *d, const double *h, int n, cudaStream_t s) {
    return cuda_check(cudaMemcpyAsync(d, h, n * sizeof(double), cudaMemcpyHostToDevice, s), "H2D scalars");
}

#define TRY(x)                  \
    do {                        \
        int rc_ = (x);          \
        if (rc_) return rc_;    \
    } while (0)

struct CoreOut {
    int iters = 0, recomputes = 0, status = 0;
    int status_rhs[kNS];
    double relres[kNS];
};

// Per-RHS CG coefficient history for the Lanczos estimate of the extreme
// eigenvalues of A (the "cond" module of App. F): alpha_j = rr_j / <p_j, A p_j>,
// beta_j = rr_{j+1} / rr_j.
struct Lanczos {
    std::vector<double> alpha[kNS], beta[kNS];
    void add(int nv, const double *act, const double *rr, const double *pq, const double *rn) {
        for (int v = 0; v < nv; ++v) {
            if (act[v] == 0.0 || pq[v] <= 0.0 || rr[v] <= 0.0) continue;
            alpha[v].push_back(rr[v] / pq[v]);
            beta[v].push_back(rn[v] / rr[v]);
        }
    }
};

// number of eigenvalues below x of the symmetric tridiagonal (d, e) (Sturm count)
static int sturm_count(const std::vector<double> &d, const std::vector<double> &e, double x) {
    int cnt = 0;
    double q = 1.0;
    for (size_t i = 0; i < d.size(); ++i) {
        const double off = i ? e[i - 1] * e[i - 1] : 0.0;
        q = (d[i] - x) - (i ? off / q : 0.0);
        if (q == 0.0) q = -1e-300;
        if (q < 0) ++cnt;
    }
    return cnt;
}

// smallest and largest eigenvalue of the Lanczos matrix built from the CG
// coefficients: diagonal 1/alpha_j + beta_{j-1}/alpha_{j-1}, off-diagonal
// sqrt(beta_j)/alpha_j; bisection on the Gershgorin interval.
static void lanczos_extremes(const std::vector<double> &al, const std::vector<double> &be, double &lmin,
                             double &lmax) {
    const size_t k = al.size();
    lmin = lmax = 0.0;
    if (k == 0) return;
    std::vector<double> d(k), e(k > 1 ? k - 1 : 0);
    for (size_t j = 0; j < k; ++j) {
        d[j] = 1.0 / al[j] + (j ? be[j - 1] / al[j - 1] : 0.0);
        if (j + 1 < k) e[j] = sqrt(be[j]) / al[j];
    }
    double lo = 1e300, hi = -1e300;
    for (size_t j = 0; j < k; ++j) {
        const double r = (j ? fabs(e[j - 1]) : 0.0) + (j + 1 < k ? fabs(e[j]) : 0.0);
        lo = fmin(lo, d[j] - r);
        hi = fmax(hi, d[j] + r);
    }
    double a = lo, b = hi;
    for (int it = 0; it < 200 && b - a > 1e-15 * fmax(fabs(a), fabs(b)); ++it) {
        const double m = 0.5 * (a + b);
        if (sturm_count(d, e, m) >= 1) b = m; else a = m;
    }
    lmin = 0.5 * (a + b);
    a = lo;
    b = hi;
    for (int it = 0; it < 200 && b - a > 1e-15 * fmax(fabs(a), fabs(b)); ++it) {
        const double m = 0.5 * (a + b);
        if (sturm_count(d, e, m) >= (int)k) b = m; else a = m;
    }
    lmax = 0.5 * (a + b);
}

// The CG operator: D^dag D through the operator scratch, or A itself for the
// hermitian positive definite Laplace kinds.
static int apply_A(const dirac_op *op, const void *in, void *out, double m0, cudaStream_t s) {
    return op_apply_cg(op, in, out, m0, s);
}

// q = D^dag D p through the operator scratch, with pq = Re <p, q> per RHS.
// The step length must match the q that is subtracted from r: |D p|^2 from
// the intermediate would save one vector read, but it differs from <p, q> by
// the rounding of D p and of q, and in FP32 the gap between the updated and
// the true residual then grows until the 1% rule stops the solve (measured on
// staggered solves at cond ~ 2e3).
static int apply_A_pq(const dirac_op *op, const void *p, void *q, double *pq, double m0, cudaStream_t s) {
    int rc = op_apply(op, p, is_laplace(op->kind) ? q : op->scratch, m0, +1, s);
    if (!rc && !is_laplace(op->kind)) rc = op_apply(op, op->scratch, q, m0, -1, s);
    if (!rc) rc = blas_dot_re(op, op->prec, p, q, pq, s);
    return rc;
}

// CG on A x = rhs (A = D^dag D), x in/out.  Uses ws vectors 0..2.
static int cg_core(const dirac_op *op, const void *rhs, void *x, double m0, double tol, int maxit, int every,
                   CoreOut &out, cudaStream_t s, Lanczos *lan = nullptr) {
    Ws w;
    TRY(get_ws(op, w));
    const int nv = op->nv;
    const dirac_prec p = op->prec;
    void *r = w.v[0], *pv = w.v[1], *q = w.v[2];
    double nb[kNS], rr[kNS], act[kNS], rrt[kNS];
    TRY(blas_norm2(op, p, rhs, w.nb, s));
    TRY(to_host(nb, w.nb, nv, s));
    // r = rhs - A x
    TRY(apply_A(op, x, q, m0, s));
    TRY(blas_axpby(op, p, r, rhs, nullptr, 1.0, q, nullptr, -1.0, w.rr, s));
    TRY(blas_axpby(op, p, pv, r, nullptr, 1.0, nullptr, nullptr, 0.0, nullptr, s));
    TRY(to_host(rr, w.rr, nv, s));
    int nact = 0;
    for (int v = 0; v < nv; ++v) {
        const bool conv = nb[v] == 0.0 || sqrt(rr[v]) < tol * sqrt(nb[v]);
        act[v] = conv ? 0.0 : 1.0;
        out.status_rhs[v] = conv ? DIRAC_OK : DIRAC_NOT_CONVERGED;
        out.relres[v] = nb[v] > 0 ? sqrt(rr[v] / nb[v]) : 0.0;
        nact += !conv;
    }
    TRY(to_dev(w.act, act, nv, s));
    out.status = DIRAC_OK;
    int it = 0;
    while (nact > 0) {
        ++it;
        TRY(apply_A_pq(op, pv, q, w.pq, m0, s));
        cg_alpha_kernel<<<1, kNS, 0, s>>>(nv, w.rr, w.pq, w.act, w.alpha);
        TRY(blas_axpby(op, p, r, r, nullptr, 1.0, q, w.alpha, -1.0, w.rr_new, s));
        double rn[kNS], pq[kNS], rro[kNS];
        if (lan) {
            TRY(cuda_check(cudaMemcpyAsync(pq, w.pq, nv * sizeof(double), cudaMemcpyDeviceToHost, s), "D2H"));
            TRY(cuda_check(cudaMemcpyAsync(rro, w.rr, nv * sizeof(double), cudaMemcpyDeviceToHost, s), "D2H"));
        }
        TRY(to_host(rn, w.rr_new, nv, s));
        if (lan) lan->add(nv, act, rro, pq, rn);
        bool all_pass = true, finite = true;
        for (int v = 0; v < nv; ++v) {
            if (!isfinite(rn[v])) finite = false;
            if (act[v] != 0.0 && !(sqrt(rn[v]) < tol * sqrt(nb[v]))) all_pass = false;
        }
        if (!finite) {
            out.status = DIRAC_NONFINITE;
            break;
        }
        const bool recompute = it % every == 0 || all_pass || it >= maxit;
        if (recompute) {
            // the solution update is needed now; otherwise it is fused with p below
            TRY(blas_axpby(op, p, x, x, nullptr, 1.0, pv, w.alpha, 1.0, nullptr, s));
            out.recomputes++;
            TRY(apply_A(op, x, q, m0, s));
            TRY(blas_axpby(op, p, r, rhs, nullptr, 1.0, q, nullptr, -1.0, w.rr_new, s));
            TRY(to_host(rrt, w.rr_new, nv, s));
            bool stagnated = false;
            nact = 0;
            for (int v = 0; v < nv; ++v) {
                out.relres[v] = nb[v] > 0 ? sqrt(rrt[v] / nb[v]) : 0.0;
                if (act[v] == 0.0) continue;
                if (sqrt(rrt[v]) < tol * sqrt(nb[v])) {
                    act[v] = 0.0;
                    out.status_rhs[v] = DIRAC_OK;
                    continue;
                }
                const double disc = fabs(sqrt(rn[v]) - sqrt(rrt[v])) / fmax(sqrt(rrt[v]), 1e-300);
                if (disc > 0.01) stagnated = true;
                ++nact;
            }
            TRY(to_dev(w.act, act, nv, s));
            if (nact == 0) break;
            if (stagnated) {
                out.status = DIRAC_STAGNATED;
                for (int v = 0; v < nv; ++v)
                    if (act[v] != 0.0) out.status_rhs[v] = DIRAC_STAGNATED;
                break;
            }
            if (it >= maxit) {
                out.status = DIRAC_NOT_CONVERGED;
                break;
            }
        }
        cg_beta_kernel<<<1, kNS, 0, s>>>(nv, w.rr_new, w.rr, w.act, w.beta);
        if (recompute) TRY(blas_axpby(op, p, pv, r, nullptr, 1.0, pv, w.beta, 1.0, nullptr, s));
        else TRY(blas_update_xp(op, p, x, pv, r, w.alpha, w.beta, s));   // x += alpha p; p = r + beta p
    }
    out.iters = it;
    TRY(launch_check("cg coefficient kernels"));
    return DIRAC_OK;
}

// BiCGstab on D x = b, x in/out.  Uses ws vectors 0..4.
static int bicgstab_core(const dirac_op *op, const void *b, void *x, double m0, double tol, int maxit, int every,
                         CoreOut &out, cudaStream_t s) {
    Ws w;
    TRY(get_ws(op, w));
    const int nv = op->nv;
    const dirac_prec p = op->prec;
    void *r = w.v[0], *rh = w.v[1], *pv = w.v[2], *vv = w.v[3], *t = w.v[4];
    double nb[kNS], rr[kNS], act[kNS], brk[kNS];
    TRY(blas_norm2(op, p, b, w.nb, s));
    TRY(to_host(nb, w.nb, nv, s));
    TRY(op_apply(op, x, t, m0, +1, s));
    TRY(blas_axpby(op, p, r, b, nullptr, 1.0, t, nullptr, -1.0, w.rr, s));
    TRY(blas_axpby(op, p, rh, r, nullptr, 1.0, nullptr, nullptr, 0.0, nullptr, s));
    TRY(cuda_check(cudaMemsetAsync(pv, 0, op->vec_bytes, s), "memset"));
    TRY(cuda_check(cudaMemsetAsync(vv, 0, op->vec_bytes, s), "memset"));
    TRY(to_host(rr, w.rr, nv, s));
    double ones[2 * kNS];
    for (int i = 0; i < 2 * kNS; ++i) ones[i] = (i & 1) ? 0.0 : 1.0;
    TRY(to_dev(w.rho, ones, 2 * nv, s));
    TRY(to_dev(w.alpha, ones, 2 * nv, s));
    TRY(to_dev(w.omega, ones, 2 * nv, s));
    int nact = 0;
    for (int v = 0; v < nv; ++v) {
        const bool conv = nb[v] == 0.0 || sqrt(rr[v]) < tol * sqrt(nb[v]);
        act[v] = conv ? 0.0 : 1.0;
        brk[v] = 0.0;
        out.status_rhs[v] = conv ? DIRAC_OK : DIRAC_NOT_CONVERGED;
        out.relres[v] = nb[v] > 0 ? sqrt(rr[v] / nb[v]) : 0.0;
        nact += !conv;
    }
    TRY(to_dev(w.act, act, nv, s));
    double *brk_d = w.c3;   // breakdown flags
    TRY(to_dev(brk_d, brk, nv, s));
    out.status = DIRAC_OK;
    int it = 0;
    while (nact > 0) {
        ++it;
        TRY(blas_dot(op, p, rh, r, w.rho_new, s));
        bicg_beta_kernel<<<1, kNS, 0, s>>>(nv, w.rho_new, w.rho, w.alpha, w.omega, w.act, w.beta, w.c2, brk_d);
        // p = r + beta p - beta omega v
        TRY(blas_axpby(op, p, pv, pv, w.beta, 1.0, vv, w.c2, 1.0, nullptr, s));
        TRY(blas_axpby(op, p, pv, pv, nullptr, 1.0, r, nullptr, 1.0, nullptr, s));
        TRY(op_apply(op, pv, vv, m0, +1, s));
        TRY(blas_dot(op, p, rh, vv, w.pq, s));
        bicg_alpha_kernel<<<1, kNS, 0, s>>>(nv, w.rho_new, w.pq, w.act, w.alpha);
        // s = r - alpha v (in r)
        TRY(blas_axpby(op, p, r, r, nullptr, 1.0, vv, w.alpha, -1.0, nullptr, s));
        TRY(op_apply(op, r, t, m0, +1, s));
        TRY(blas_dot(op, p, t, r, w.c1, s));
        TRY(blas_norm2(op, p, t, w.tt, s));
        bicg_omega_kernel<<<1, kNS, 0, s>>>(nv, w.c1, w.tt, w.act, w.omega, w.rho_new, w.rho, brk_d, w.act);
        // x += alpha p + omega s
        TRY(blas_axpby(op, p, x, x, nullptr, 1.0, pv, w.alpha, 1.0, nullptr, s));
        TRY(blas_axpby(op, p, x, x, nullptr, 1.0, r, w.omega, 1.0, nullptr, s));
        // r = s - omega t
        TRY(blas_axpby(op, p, r, r, nullptr, 1.0, t, w.omega, -1.0, w.rr_new, s));
        double rn[kNS];
        TRY(to_host(rn, w.rr_new, nv, s));
        TRY(to_host(act, w.act, nv, s));   // breakdown may have frozen some
        bool all_pass = true, finite = true;
        for (int v = 0; v < nv; ++v) {
            if (!isfinite(rn[v])) finite = false;
            if (act[v] != 0.0 && !(sqrt(rn[v]) < tol * sqrt(nb[v]))) all_pass = false;
        }
        if (!finite) {
            out.status = DIRAC_NONFINITE;
            break;
        }
        nact = 0;
        for (int v = 0; v < nv; ++v) nact += act[v] != 0.0;
        if (it % every == 0 || all_pass || it >= maxit || nact == 0) {
            out.recomputes++;
            TRY(op_apply(op, x, t, m0, +1, s));
            TRY(blas_axpby(op, p, r, b, nullptr, 1.0, t, nullptr, -1.0, w.rr_new, s));
            double rrt[kNS];
            TRY(to_host(rrt, w.rr_new, nv, s));
            bool stagnated = false;
            nact = 0;
            for (int v = 0; v < nv; ++v) {
                out.relres[v] = nb[v] > 0 ? sqrt(rrt[v] / nb[v]) : 0.0;
                if (sqrt(rrt[v]) < tol * sqrt(nb[v])) {
                    if (act[v] != 0.0 || out.status_rhs[v] != DIRAC_OK) out.status_rhs[v] = DIRAC_OK;
                    act[v] = 0.0;
                    continue;
                }
                if (act[v] == 0.0) continue;
                const double disc = fabs(sqrt(rn[v]) - sqrt(rrt[v])) / fmax(sqrt(rrt[v]), 1e-300);
                if (disc > 0.01) stagnated = true;
                ++nact;
            }
            TRY(to_dev(w.act, act, nv, s));
            if (nact == 0) break;
            if (stagnated) {
                out.status = DIRAC_STAGNATED;
                break;
            }
            if (it >= maxit) {
                out.status = DIRAC_NOT_CONVERGED;
                break;
            }
        }
    }
    TRY(to_host(brk, brk_d, nv, s));
    for (int v = 0; v < nv; ++v)
        if (brk[v] != 0.0 && out.status_rhs[v] != DIRAC_OK) {
            out.status_rhs[v] = DIRAC_BREAKDOWN;
            if (out.status == DIRAC_OK) out.status = DIRAC_BREAKDOWN;
        }
    for (int v = 0; v < nv; ++v)
        if (out.status_rhs[v] == DIRAC_NOT_CONVERGED && out.status != DIRAC_OK) out.status_rhs[v] = out.status;
    out.iters = it;
    TRY(launch_check("bicgstab coefficient kernels"));
    return DIRAC_OK;
}

// previous sloppy |r|^2 expressed in the new scaling (ratio = 0 restarts p)
__global__ void scale_rr_kernel(int nv, const double *ratio, double *rr) {
    const int v = threadIdx.x;
    if (v >= nv) return;
    rr[v] *= ratio[2 * v] * ratio[2 * v];
}

__global__ void inverse_kernel(int nv, const double *c, double *inv) {
    const int v = threadIdx.x;
    if (v >= nv) return;
    inv[2 * v] = c[2 * v] != 0.0 ? 1.0 / c[2 * v] : 0.0;
    inv[2 * v + 1] = 0.0;
}

// Mixed-precision CG on A x = rhs (A = D^dag D) with reliable updates: the
// Krylov iteration runs in the precision of `lo` on the residual scaled to
// unit norm per RHS; whenever the sloppy residual has dropped by `delta`
// since the last update (or looks converged, or at maxit) the accumulated
// correction is added to x and r = rhs - A x is recomputed in the precision
// of `hi`, rescaled, and the iteration continues with its search direction
// (rescaled) instead of restarting.  Converged RHS are frozen.
// Workspace: hi vectors 0..1, lo vectors 0..3.
static int cg_reliable(const dirac_op *hi, const dirac_op *lo, const void *rhs, void *x, double m0, double tol,
                       int maxit, double delta, CoreOut &out, Lanczos *lan, cudaStream_t s, int give_up = 30) {
    Ws wh, wl;
    TRY(get_ws(hi, wh));
    TRY(get_ws(lo, wl));
    const int nv = hi->nv;
    const dirac_prec ph = hi->prec, pl = lo->prec;
    void *rh = wh.v[0], *th = wh.v[1];
    void *rs = wl.v[0], *ps = wl.v[1], *qs = wl.v[2], *ys = wl.v[3];
    double *sig = wh.c1, *ratio = wh.c3, *inv = wh.omega;
    double nb[kNS], rrt[kNS], act[kNS], rmax[kNS], prev_true[kNS], best[kNS], best_true[kNS];
    int slow[kNS], since_best[kNS];
    // sloppy iterations without a new residual minimum that force an update
    // (CG residual norms are not monotone, so this is only a safety net)
    const int kStall = 100;
    TRY(blas_norm2(hi, ph, rhs, wh.nb, s));
    TRY(to_host(nb, wh.nb, nv, s));
    // true residual and first scaling
    TRY(apply_A(hi, x, th, m0, s));
    TRY(blas_axpby(hi, ph, rh, rhs, nullptr, 1.0, th, nullptr, -1.0, wh.rr, s));
    TRY(to_host(rrt, wh.rr, nv, s));
    int nact = 0;
    for (int v = 0; v < nv; ++v) {
        const bool conv = nb[v] == 0.0 || sqrt(rrt[v]) < tol * sqrt(nb[v]);
        act[v] = conv ? 0.0 : 1.0;
        out.status_rhs[v] = conv ? DIRAC_OK : DIRAC_NOT_CONVERGED;
        out.relres[v] = nb[v] > 0 ? sqrt(rrt[v] / nb[v]) : 0.0;
        prev_true[v] = best_true[v] = sqrt(rrt[v]);
        slow[v] = 0;
        nact += !conv;
    }
    TRY(to_dev(wh.act, act, nv, s));
    TRY(to_dev(wl.act, act, nv, s));
    // sloppy vectors carry the residual scaled to unit rms per component (not
    // unit norm): FP16 would otherwise hold most components near its
    // subnormal range on large lattices
    const double unit = sqrt((double)hi->rows);
    coef_from_norm_kernel<<<1, kNS, 0, s>>>(nv, wh.rr, wh.act, sig, 1, unit);
    TRY(blas_axpby(hi, ph, th, rh, sig, 1.0, nullptr, nullptr, 0.0, nullptr, s));
    TRY(blas_convert(hi, th, ph, rs, pl, s));
    TRY(blas_axpby(lo, pl, ps, rs, nullptr, 1.0, nullptr, nullptr, 0.0, nullptr, s));
    TRY(cuda_check(cudaMemsetAsync(ys, 0, lo->vec_bytes, s), "memset"));
    TRY(blas_norm2(lo, pl, rs, wl.rr, s));
    double rr0[kNS];
    TRY(to_host(rr0, wl.rr, nv, s));
    for (int v = 0; v < nv; ++v) {
        rmax[v] = best[v] = sqrt(rr0[v]);
        since_best[v] = 0;
    }
    double sig_h[kNS];
    for (int v = 0; v < nv; ++v) sig_h[v] = (act[v] != 0.0 && rrt[v] > 0) ? unit / sqrt(rrt[v]) : 0.0;
    out.status = DIRAC_OK;
    int it = 0;
    while (nact > 0) {
        ++it;
        TRY(apply_A_pq(lo, ps, qs, wl.pq, m0, s));
        cg_alpha_kernel<<<1, kNS, 0, s>>>(nv, wl.rr, wl.pq, wl.act, wl.alpha);
        TRY(blas_axpby(lo, pl, rs, rs, nullptr, 1.0, qs, wl.alpha, -1.0, wl.rr_new, s));
        double rn[kNS], pq[kNS], rro[kNS];
        if (lan) {
            TRY(cuda_check(cudaMemcpyAsync(pq, wl.pq, nv * sizeof(double), cudaMemcpyDeviceToHost, s), "D2H"));
            TRY(cuda_check(cudaMemcpyAsync(rro, wl.rr, nv * sizeof(double), cudaMemcpyDeviceToHost, s), "D2H"));
        }
        TRY(to_host(rn, wl.rr_new, nv, s));
        if (lan) lan->add(nv, act, rro, pq, rn);
        bool trigger = it >= maxit, finite = true;
        bool stalled[kNS];
        for (int v = 0; v < nv; ++v) {
            stalled[v] = false;
            if (!isfinite(rn[v])) finite = false;
            if (act[v] == 0.0) continue;
            const double r = sqrt(rn[v]);
            if (r < best[v]) {
                best[v] = r;
                since_best[v] = 0;
            } else if (++since_best[v] >= kStall) {
                trigger = true;   // the sloppy recurrence stopped improving: refresh it
            }
            if (r < delta * rmax[v] || r < tol * sqrt(nb[v]) * sig_h[v]) trigger = true;
        }
        if (!finite) {
            out.status = DIRAC_NONFINITE;
            break;
        }
        if (trigger) {
            out.recomputes++;
            TRY(blas_axpby(lo, pl, ys, ys, nullptr, 1.0, ps, wl.alpha, 1.0, nullptr, s));
            // x += y / sigma, then the true residual in the high precision
            inverse_kernel<<<1, kNS, 0, s>>>(nv, sig, inv);
            TRY(blas_convert(lo, ys, pl, th, ph, s));
            TRY(blas_axpby(hi, ph, x, x, nullptr, 1.0, th, inv, 1.0, nullptr, s));
            TRY(apply_A(hi, x, th, m0, s));
            TRY(blas_axpby(hi, ph, rh, rhs, nullptr, 1.0, th, nullptr, -1.0, wh.rr, s));
            TRY(to_host(rrt, wh.rr, nv, s));
            nact = 0;
            bool stagnated = false;
            for (int v = 0; v < nv; ++v) {
                out.relres[v] = nb[v] > 0 ? sqrt(rrt[v] / nb[v]) : 0.0;
                if (act[v] == 0.0) continue;
                if (!isfinite(rrt[v])) {
                    out.status = DIRAC_NONFINITE;
                    return DIRAC_OK;
                }
                if (sqrt(rrt[v]) < tol * sqrt(nb[v])) {
                    act[v] = 0.0;
                    out.status_rhs[v] = DIRAC_OK;
                    continue;
                }
                // the true residual grew across the segment: the sloppy search
                // direction is no longer useful, restart it below
                stalled[v] = stalled[v] || sqrt(rrt[v]) > prev_true[v];
                // give up when give_up updates in a row failed to halve the best true residual
                if (sqrt(rrt[v]) < 0.5 * best_true[v]) {
                    best_true[v] = sqrt(rrt[v]);
                    slow[v] = 0;
                } else if (++slow[v] >= give_up) {
                    stagnated = true;
                }
                prev_true[v] = sqrt(rrt[v]);
                ++nact;
            }
            TRY(to_dev(wh.act, act, nv, s));
            TRY(to_dev(wl.act, act, nv, s));
            if (nact == 0) break;
            if (stagnated) {
                out.status = DIRAC_STAGNATED;
                for (int v = 0; v < nv; ++v)
                    if (act[v] != 0.0) out.status_rhs[v] = DIRAC_STAGNATED;
                break;
            }
            if (it >= maxit) {
                out.status = DIRAC_NOT_CONVERGED;
                break;
            }
            // rescale: r_s = sigma_new r, p_s *= sigma_new / sigma_old (0 = restart a
            // stalled direction), y_s = 0
            double rat[2 * kNS];
            for (int v = 0; v < nv; ++v) {
                const double sn = (act[v] != 0.0 && rrt[v] > 0) ? unit / sqrt(rrt[v]) : 0.0;
                rat[2 * v] = (stalled[v] || sig_h[v] == 0.0) ? 0.0 : sn / sig_h[v];
                rat[2 * v + 1] = 0.0;
            }
            TRY(to_dev(ratio, rat, 2 * nv, s));
            coef_from_norm_kernel<<<1, kNS, 0, s>>>(nv, wh.rr, wh.act, sig, 1, unit);
            scale_rr_kernel<<<1, kNS, 0, s>>>(nv, ratio, wl.rr);
            TRY(blas_axpby(hi, ph, th, rh, sig, 1.0, nullptr, nullptr, 0.0, nullptr, s));
            TRY(blas_convert(hi, th, ph, rs, pl, s));
            TRY(blas_axpby(lo, pl, ps, ps, ratio, 1.0, nullptr, nullptr, 0.0, nullptr, s));
            TRY(cuda_check(cudaMemsetAsync(ys, 0, lo->vec_bytes, s), "memset"));
            TRY(blas_norm2(lo, pl, rs, wl.rr_new, s));
            TRY(to_host(rn, wl.rr_new, nv, s));
            for (int v = 0; v < nv; ++v) {
                rmax[v] = best[v] = sqrt(rn[v]);
                since_best[v] = 0;
                sig_h[v] = (act[v] != 0.0 && rrt[v] > 0) ? unit / sqrt(rrt[v]) : 0.0;
            }
        } else {
            for (int v = 0; v < nv; ++v) rmax[v] = fmax(rmax[v], sqrt(rn[v]));
        }
        cg_beta_kernel<<<1, kNS, 0, s>>>(nv, wl.rr_new, wl.rr, wl.act, wl.beta);
        if (trigger) TRY(blas_axpby(lo, pl, ps, rs, nullptr, 1.0, ps, wl.beta, 1.0, nullptr, s));
        else TRY(blas_update_xp(lo, pl, ys, ps, rs, wl.alpha, wl.beta, s));   // y += alpha p; p = r + beta p
    }
    out.iters = it;
    TRY(launch_check("reliable-update kernels"));
    return DIRAC_OK;
}

static double default_inner_tol(dirac_prec p) {
    switch (p) {
    case DIRAC_F32: return 1e-5;
    case DIRAC_F16: return 2e-3;
    case DIRAC_BF16: return 1e-2;
    default: return 1e-10;
    }
}

// Defect correction: outer in op precision, inner Krylov solve in inner_prec.
static int mixed_solve(const dirac_op *op, const void *b, void *x, double m0, const dirac_solve_params *prm,
                       dirac_solve_stats *st, cudaStream_t s) {
    dirac_op *lo = nullptr;
    TRY(op_inner(op, prm->inner_prec, prm->sloppy_links, &lo, s));
    Ws wh, wl;
    TRY(get_ws(op, wh));
    TRY(get_ws(lo, wl));
    const int nv = op->nv;
    const dirac_prec ph = op->prec, pl = lo->prec;
    const bool cg = prm->solver != DIRAC_BICGSTAB;
    void *rhs = wh.v[5], *r = wh.v[6], *tmp = wh.v[7];
    void *rl = wl.v[5], *el = wl.v[6];
    // rhs = D^dag b (CG on normal equations) or b
    if (prm->solver == DIRAC_CG_NORMAL) TRY(op_apply(op, b, rhs, m0, -1, s));
    else TRY(blas_axpby(op, ph, rhs, b, nullptr, 1.0, nullptr, nullptr, 0.0, nullptr, s));
    double nb[kNS], rr[kNS], act[kNS];
    TRY(blas_norm2(op, ph, rhs, wh.nb, s));
    TRY(to_host(nb, wh.nb, nv, s));
    const double itol = prm->inner_tol > 0 ? prm->inner_tol : default_inner_tol(pl);
    const int every = prm->recompute_every > 0 ? prm->recompute_every : (pl == DIRAC_F64 ? 50 : 20);
    int total = 0, outer = 0;
    st->status = DIRAC_NOT_CONVERGED;
    for (;;) {
        // r = rhs - A x (operator precision)
        if (cg) TRY(op_apply_cg(op, x, tmp, m0, s));
        else TRY(op_apply(op, x, tmp, m0, +1, s));
        TRY(blas_axpby(op, ph, r, rhs, nullptr, 1.0, tmp, nullptr, -1.0, wh.rr, s));
        TRY(to_host(rr, wh.rr, nv, s));
        st->recomputes++;
        int nact = 0;
        bool finite = true;
        for (int v = 0; v < nv; ++v) {
            if (!isfinite(rr[v])) finite = false;
            st->relres[v] = nb[v] > 0 ? sqrt(rr[v] / nb[v]) : 0.0;
            const bool conv = nb[v] == 0.0 || sqrt(rr[v]) < prm->tol * sqrt(nb[v]);
            act[v] = conv ? 0.0 : 1.0;
            st->status_per_rhs[v] = conv ? DIRAC_OK : DIRAC_NOT_CONVERGED;
            nact += !conv;
        }
        if (!finite) {
            st->status = DIRAC_NONFINITE;
            break;
        }
        if (nact == 0) {
            st->status = DIRAC_OK;
            break;
        }
        if (total >= prm->maxit) break;
        TRY(to_dev(wh.act, act, nv, s));
        // inner right-hand side r / |r| in low precision
        const double unit = sqrt((double)op->rows);   // unit rms per component (see cg_reliable)
        coef_from_norm_kernel<<<1, kNS, 0, s>>>(nv, wh.rr, wh.act, wh.c1, 1, unit);
        TRY(blas_axpby(op, ph, tmp, r, wh.c1, 1.0, nullptr, nullptr, 0.0, nullptr, s));
        TRY(blas_convert(op, tmp, ph, rl, pl, s));
        TRY(cuda_check(cudaMemsetAsync(el, 0, lo->vec_bytes, s), "memset"));
        CoreOut co;
        const int budget = prm->maxit - total;
        if (cg) TRY(cg_core(lo, rl, el, m0, itol, budget, every, co, s));
        else TRY(bicgstab_core(lo, rl, el, m0, itol, budget, every, co, s));
        total += co.iters;
        st->recomputes += co.recomputes;
        // x += |r| e
        TRY(blas_convert(op, el, pl, tmp, ph, s));
        coef_from_norm_kernel<<<1, kNS, 0, s>>>(nv, wh.rr, wh.act, wh.c1, 0, unit);
        TRY(blas_axpby(op, ph, x, x, nullptr, 1.0, tmp, wh.c1, 1.0, nullptr, s));
        ++outer;
        if (co.iters == 0) break;   // inner solver made no progress
    }
    st->iters = total;
    st->outer_iters = outer;
    return DIRAC_OK;
}

static void lanczos_stats(const Lanczos &lan, int nv, dirac_solve_stats *st) {
    for (int v = 0; v < nv; ++v) lanczos_extremes(lan.alpha[v], lan.beta[v], st->lambda_min[v], st->lambda_max[v]);
}

static int reliable_solve(const dirac_op *op, const void *b, void *x, double m0, const dirac_solve_params *prm,
                          dirac_solve_stats *st, cudaStream_t s) {
    dirac_op *lo = nullptr;
    TRY(op_inner(op, prm->inner_prec, prm->sloppy_links, &lo, s));
    Ws w;
    TRY(get_ws(op, w));
    void *rhs = w.v[5];
    if (prm->solver == DIRAC_CG_NORMAL) TRY(op_apply(op, b, rhs, m0, -1, s));
    else TRY(blas_axpby(op, op->prec, rhs, b, nullptr, 1.0, nullptr, nullptr, 0.0, nullptr, s));
    CoreOut co;
    Lanczos lan;
    const double delta = prm->delta > 0 ? prm->delta : 0.1;
    const bool half = prm->inner_prec == DIRAC_BF16 || prm->inner_prec == DIRAC_F16;
    const bool adaptive = prm->mixed_mode == DIRAC_MIXED_ADAPTIVE && half && op->prec == DIRAC_F64;
    // adaptive: the 16-bit iteration runs while reliable updates keep halving
    // the true residual (2 misses in a row end it), then an FP32 iteration
    // continues from the current solution
    const auto t16 = std::chrono::steady_clock::now();
    TRY(cg_reliable(op, lo, rhs, x, m0, prm->tol, prm->maxit, delta, co, &lan, s, adaptive ? 2 : 30));
    int iters = co.iters, updates = co.recomputes;
    if (half) {   // cg_reliable reads the residual norms on the host every iteration: the wall time is the GPU's
        st->iters_16bit = co.iters;
        st->seconds_16bit = std::chrono::duration<double>(std::chrono::steady_clock::now() - t16).count();
    }
    if (adaptive && co.status == DIRAC_STAGNATED && co.iters < prm->maxit) {
        dirac_op *lo32 = nullptr;
        TRY(op_inner(op, DIRAC_F32, DIRAC_LINKS_NATIVE, &lo32, s));
        CoreOut co2;
        Lanczos lan2;
        TRY(cg_reliable(op, lo32, rhs, x, m0, prm->tol, prm->maxit - co.iters, delta, co2, &lan2, s));
        co = co2;
        lan = lan2;
        iters += co2.iters;
        updates += co2.recomputes;
    }
    st->iters = iters;
    st->outer_iters = updates;
    st->recomputes = updates;
    st->status = co.status;
    bool all = true;
    for (int v = 0; v < op->nv; ++v) {
        st->status_per_rhs[v] = co.status_rhs[v];
        st->relres[v] = co.relres[v];
        all &= co.status_rhs[v] == DIRAC_OK;
    }
    if (all) st->status = DIRAC_OK;
    else if (st->status == DIRAC_OK) st->status = DIRAC_NOT_CONVERGED;
    lanczos_stats(lan, op->nv, st);
    return DIRAC_OK;
}

static int plain_solve(const dirac_op *op, const void *b, void *x, double m0, const dirac_solve_params *prm,
                       dirac_solve_stats *st, cudaStream_t s) {
    Ws w;
    TRY(get_ws(op, w));
    const int every = prm->recompute_every > 0 ? prm->recompute_every : (op->prec == DIRAC_F64 ? 50 : 20);
    CoreOut co;
    Lanczos lan;
    if (prm->solver == DIRAC_CG_NORMAL) {
        void *rhs = w.v[5];
        TRY(op_apply(op, b, rhs, m0, -1, s));
        TRY(cg_core(op, rhs, x, m0, prm->tol, prm->maxit, every, co, s, &lan));
        lanczos_stats(lan, op->nv, st);
    } else if (prm->solver == DIRAC_CG_HPD) {
        TRY(cg_core(op, b, x, m0, prm->tol, prm->maxit, every, co, s, &lan));
        lanczos_stats(lan, op->nv, st);
    } else {
        TRY(bicgstab_core(op, b, x, m0, prm->tol, prm->maxit, every, co, s));
    }
    st->iters = co.iters;
    st->outer_iters = 0;
    st->recomputes = co.recomputes;
    st->status = co.status;
    for (int v = 0; v < op->nv; ++v) {
        st->status_per_rhs[v] = co.status_rhs[v];
        st->relres[v] = co.relres[v];
    }
    bool all = true;
    for (int v = 0; v < op->nv; ++v) all &= co.status_rhs[v] == DIRAC_OK;
    if (all) st->status = DIRAC_OK;
    else if (st->status == DIRAC_OK) st->status = DIRAC_NOT_CONVERGED;
    return DIRAC_OK;
}

int solve(const dirac_op *op, const void *b, void *x, double m0, const dirac_solve_params *prm,
          dirac_solve_stats *st_user, cudaStream_t s) {
    auto t0 = std::chrono::steady_clock::now();
    dirac_solve_stats st;
    memset(&st, 0, sizeof(st));
    int rc;
    if (prm->inner_prec == op->prec) rc = plain_solve(op, b, x, m0, prm, &st, s);
    else if (prm->solver != DIRAC_BICGSTAB && prm->mixed_mode != DIRAC_MIXED_RESTART)
        rc = reliable_solve(op, b, x, m0, prm, &st, s);
    else rc = mixed_solve(op, b, x, m0, prm, &st, s);
    if (rc) return rc;
    // true residual ||b - D x|| / ||b|| (||b - A x|| / ||b|| for CG_HPD)
    Ws w;
    TRY(get_ws(op, w));
    if (prm->solver == DIRAC_CG_HPD) TRY(op_apply_cg(op, x, w.v[7], m0, s));
    else TRY(op_apply(op, x, w.v[7], m0, +1, s));
    TRY(blas_axpby(op, op->prec, w.v[6], b, nullptr, 1.0, w.v[7], nullptr, -1.0, w.rr, s));
    TRY(blas_norm2(op, op->prec, b, w.nb, s));
    double rr[kNS], nb[kNS];
    TRY(to_host(rr, w.rr, op->nv, s));
    TRY(to_host(nb, w.nb, op->nv, s));
    for (int v = 0; v < op->nv; ++v) st.true_relres[v] = nb[v] > 0 ? sqrt(rr[v] / nb[v]) : 0.0;
    st.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (st_user) *st_user = st;
    return st.status;
}

}  // namespace dgb

extern "C" int dirac_solve(const dirac_op *op, const void *b, void *x, double m0, const dirac_solve_params *params,
                           dirac_solve_stats *stats, void *stream) {
    if (!op || !params || !b || !x) return DIRAC_ERR_INVALID_ARG;
    if (((uintptr_t)b & 15) || ((uintptr_t)x & 15)) return DIRAC_ERR_ALIGNMENT;
    if (params->solver != DIRAC_CG_NORMAL && params->solver != DIRAC_BICGSTAB && params->solver != DIRAC_CG_HPD)
        return DIRAC_ERR_INVALID_ARG;
    if (params->inner_prec < DIRAC_F64 || params->inner_prec > DIRAC_F16) return DIRAC_ERR_UNSUPPORTED_PREC;
    if (!(params->tol > 0) || params->maxit < 1) return DIRAC_ERR_INVALID_ARG;
    if (dgb::is_laplace(op->kind)) {   // A is already hpd; FP64 / FP32 only
        if (params->solver == DIRAC_CG_NORMAL) return DIRAC_ERR_INVALID_ARG;
        if (params->inner_prec != DIRAC_F64 && params->inner_prec != DIRAC_F32) return DIRAC_ERR_UNSUPPORTED_PREC;
    }
    if (params->mixed_mode != DIRAC_MIXED_RELIABLE && params->mixed_mode != DIRAC_MIXED_RESTART &&
        params->mixed_mode != DIRAC_MIXED_ADAPTIVE)
        return DIRAC_ERR_INVALID_ARG;
    if (params->delta < 0 || params->delta >= 1) return DIRAC_ERR_INVALID_ARG;
    if (params->sloppy_links != DIRAC_LINKS_NATIVE && params->sloppy_links != DIRAC_LINKS_F32)
        return DIRAC_ERR_INVALID_ARG;
    return dgb::solve(op, b, x, m0, params, stats, (cudaStream_t)stream);
}
