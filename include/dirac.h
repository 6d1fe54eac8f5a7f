/*
 * dirac.h -- C ABI of the GB300 multi-RHS lattice Dirac operator library.
 *
 * Operators and solvers of Duerr, "Fast and flexible implementations of
 * Wilson, Brillouin and Susskind fermions in lattice QCD", arXiv:2112.14640:
 *   Wilson     D_W  Eq. (app_wils),   9-point stencil, spin projection (App. A)
 *   Brillouin  D_B  Eq. (app_bril),  81-point stencil on path-averaged links
 *                                     W_s(n) (Tab. off-axis)
 *   staggered  D_S  Eq. (def_stag),   9-point stencil with eta phases
 * each applied to N_v right-hand sides at once (Sec. 1: b and u are n x N_v
 * matrices), plus CG on D^dag D, BiCGstab on D (Sec. 9) and a mixed-precision
 * defect-correction driver around them (Sec. 9, last paragraph).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Lattice: dims = {Nx, Ny, Nz, Nt}; site n = ((t*Nz + z)*Ny + y)*Nx + x.
 * Direction mu = 0..3 is x, y, z, t (the paper's mu = 1..4).
 * Complex numbers are stored interleaved (re, im) in the element type of the
 * precision: F64 double, F32 float, BF16 __nv_bfloat16, F16 __half.
 * Layouts (C order, RHS index v innermost -- the paper's NvNsNc / NvNc, Sec. 2):
 *   gauge links       U  [site][mu][a][b]         (U_mu(n)_{ab}, transporter n+mu -> n)
 *   Wilson-type vector   [site][colour][spin][v]   spin in the chiral basis of App. A
 *   staggered vector     [site][colour][v]
 * All pointers are DEVICE pointers unless a name says host; the caller owns
 * every buffer it passes and the library never frees them.  Vector buffers
 * must be 16-byte aligned.  Work is enqueued on the CUDA stream given as
 * `stream` (a cudaStream_t; NULL = legacy default stream) and is asynchronous
 * unless stated otherwise.
 *
 * Return codes: 0 = success; negative = error (nothing was launched);
 * positive = solver outcome (the solution buffer holds the last iterate).
 */
#ifndef DIRAC_H
#define DIRAC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Operator kinds.  The three Dirac operators, and the Laplace operators
 * A = -1/2 Lap + m^2/2 of Secs. 6 and 7 (the paper's wlap, blap, wsuv and
 * bsuv routines, App. F): the standard 9-point Laplacian, Eq. (app_wlap),
 * and the Brillouin 81-point Laplacian, Eq. (app_blap), each on Wilson-type
 * vectors (acting trivially on the 4 spin components) or on colour-only
 * vectors (the staggered vector shape, without the staggered phases).  For
 * the Laplace kinds the m0 argument of every call is the mass m of A; A is
 * hermitian positive definite, so its dagger is A itself, and they exist in
 * F64 and F32 only. */
typedef enum {
    DIRAC_WILSON = 0, DIRAC_BRILLOUIN = 1, DIRAC_STAGGERED = 2,
    DIRAC_WLAP = 3,   /* -1/2 Lap_std + m^2/2 on Wilson-type vectors */
    DIRAC_BLAP = 4,   /* -1/2 Lap_bri + m^2/2 on Wilson-type vectors (builds W) */
    DIRAC_WSUV = 5,   /* -1/2 Lap_std + m^2/2 on colour-only vectors */
    DIRAC_BSUV = 6    /* -1/2 Lap_bri + m^2/2 on colour-only vectors (builds W) */
} dirac_kind;
typedef enum { DIRAC_F64 = 0, DIRAC_F32 = 1, DIRAC_BF16 = 2, DIRAC_F16 = 3 } dirac_prec;

enum {
    DIRAC_OK = 0,
    DIRAC_ERR_INVALID_ARG = -1,     /* null pointer, bad enum, bad geometry */
    DIRAC_ERR_UNSUPPORTED_NC = -2,  /* N_c outside the compiled set {1,2,3,4} */
    DIRAC_ERR_UNSUPPORTED_PREC = -3,
    DIRAC_ERR_ALIGNMENT = -4,       /* a vector pointer not 16-byte aligned */
    DIRAC_ERR_OOM = -5,             /* a library-owned allocation failed */
    DIRAC_ERR_CUDA = -6,            /* a CUDA call or launch failed; see stderr */
    DIRAC_ERR_DEVICE_TIMEOUT = -7,  /* a bounded device-side wait ran out */
    DIRAC_ERR_CAPACITY = -8,        /* request exceeds a fixed static capacity */
    DIRAC_NOT_CONVERGED = 1,        /* maxit reached */
    DIRAC_STAGNATED = 2,            /* updated and recomputed residual differ > 1% (Sec. 9) */
    DIRAC_BREAKDOWN = 3,            /* BiCGstab rho or omega vanished */
    DIRAC_NONFINITE = 4             /* NaN/Inf appeared in a residual */
};

/* Lattice geometry and storage precision of an operator.
 * dims   : extents, each >= 2; staggered operators need all four even
 *          (the eta phases of Eq. def_stag are periodic only then).
 * nc     : number of colours N_c: 1..8 for F64/F32 storage, 1..4 for BF16/F16
 *          (DIRAC_ERR_UNSUPPORTED_NC otherwise); 3 is the physical case and has
 *          the tuned launch variants, N_c >= 5 runs one RHS per thread.
 * nv     : number of right-hand sides N_v, 1..64.
 * bc     : +1 periodic / -1 antiperiodic per direction.  The phase multiplies
 *          U_mu(n) on the links with n_mu = N_mu - 1 before anything else
 *          (including the W links) is built from U.
 * prec   : storage precision of links, W links and the vectors passed to
 *          dirac_apply*; arithmetic is FP64 for F64 and FP32 otherwise. */
typedef struct {
    int dims[4];
    int nc;
    int nv;
    int bc[4];
    dirac_prec prec;
    int layout;        /* vector layout, DIRAC_LAYOUT_* below (0 = the paper's) */
    int link_storage;  /* DIRAC_LINKS_NATIVE: links (and W) in prec; DIRAC_LINKS_F32: FP32
                          links with 16-bit vectors (prec BF16/F16 only) */
} dirac_geom;

enum { DIRAC_LINKS_NATIVE = 0, DIRAC_LINKS_F32 = 1 };

/* Vector layouts (the RHS index v is innermost in both, so the BLAS-1 calls
 * treat every vector as a [rows][N_v] array):
 *   SITE_OUTER  Wilson-type [site][colour][spin][v], staggered [site][colour][v]
 *               -- the paper's NvNsNc / NvNc orders (Sec. 2);
 *   SITE_INNER  Wilson-type [colour][spin][site][v], staggered [colour][site][v]
 *               -- the site index moved inside the internal dofs, so that the
 *               threads of a warp, which cover consecutive sites, read one
 *               contiguous run per (colour, spin) component.
 * The gauge field handed to dirac_op_create is always [site][mu][a][b]; the
 * operator stores its own phased copy in blocks of 32 sites, the same for
 * both layouts (internal, never exposed). */
enum { DIRAC_LAYOUT_SITE_OUTER = 0, DIRAC_LAYOUT_SITE_INNER = 1 };

typedef struct dirac_op dirac_op;   /* opaque */

/* Create an operator on gauge field U (device pointer, layout above, in
 * precision u_prec = DIRAC_F64 or DIRAC_F32, no boundary phases applied).
 * The operator keeps its own copy of the phased links in geom->prec; for
 * DIRAC_BRILLOUIN, DIRAC_BLAP and DIRAC_BSUV it also builds and keeps the 80 off-centre W_s(n) of
 * Tab. off-axis (computed from U in FP64 for FP64 operators and in FP32
 * otherwise, stored in the link precision).
 * Synchronises `stream` before returning.  U may be freed afterwards. */
int dirac_op_create(dirac_kind kind, const dirac_geom *geom, const void *U,
                    dirac_prec u_prec, void *stream, dirac_op **out);

/* Replace the gauge field (same geometry); rebuilds W for the Brillouin kinds and
 * removes a clover term (dirac_op_set_clover builds it for the new field).
 * Synchronises `stream` before returning. */
int dirac_op_update_links(dirac_op *op, const void *U, dirac_prec u_prec, void *stream);

/* Clover term (Sec. 5): from now on dirac_apply, _dagger, _normal, the
 * solvers and the batched solves apply D + C (Eqs. def_wils, def_bril) with
 *   C(n) = -(c_SW / 2) sum_{mu<nu} sigma_mu,nu F_mu,nu(n),
 *   sigma_mu,nu = (i/2) [gamma_mu, gamma_nu],
 *   F_mu,nu(n) = (Q_mu,nu(n) - Q_mu,nu(n)^dag) / (8i),
 * Q_mu,nu(n) the sum of the four plaquettes of the (mu,nu) plane with a corner
 * at n, each traversed mu-step first, then nu-step (the clover-leaf field
 * strength, which the paper uses without writing it out; no trace is
 * subtracted).  V is the gauge field F is built from (device pointer, same
 * layout and precisions as U in dirac_op_create; the paper builds it from a
 * smeared field, and U itself may be passed).  Boundary phases do not enter
 * (closed loops).  C is site diagonal and commutes with gamma5, so the
 * dagger is gamma5 (D + C) gamma5 = D^dag + C.  The operator keeps C in its
 * link precision as two 2N_c x 2N_c blocks per site (FP64 arithmetic for
 * FP64 operators, FP32 otherwise); applying it adds 64 N_c^2 flops per site
 * and RHS (App. E) and 4 N_c^2 link-precision complex numbers per site of
 * traffic.  csw = 0 removes the term (V may then be NULL).  Wilson and
 * Brillouin only (DIRAC_ERR_INVALID_ARG for staggered); dirac_op_update_links
 * removes it, and dirac_force_wilson refuses an operator that carries it.
 * Synchronises `stream` before returning. */
int dirac_op_set_clover(dirac_op *op, double csw, const void *V, dirac_prec v_prec, void *stream);

/* Stout smearing of a gauge field (the fat links V the paper builds D and F
 * from, Sec. 2 and App. F; rho = 0.12, nsteps = 3 are the paper's defaults,
 * nsteps = 0 gives V = U).  Each step updates all links at once:
 *   C_mu(n) = rho sum_{nu != mu} [U_nu(n) U_mu(n+nu) U_nu(n+mu)^dag
 *                                + U_nu(n-nu)^dag U_mu(n-nu) U_nu(n-nu+mu)],
 *   Omega = C_mu(n) U_mu(n)^dag,
 *   Q = (i/2)(Omega^dag - Omega) - (i/2N_c) Tr(Omega^dag - Omega),
 *   U_mu(n) <- exp(iQ) U_mu(n)
 * (Morningstar and Peardon).  U_in, V_out: device fields [site][mu][a][b]
 * complex in prec (F64 or F32), periodic, no boundary phases (the step
 * commutes with them); they may be the same buffer.  Arithmetic in FP64;
 * exp(iQ) by scaling and squaring of the Taylor series, for any N_c.  Uses
 * one temporary field of the same size (allocated and freed here).
 * Synchronises `stream` before returning. */
int dirac_stout_smear(const void *U_in, void *V_out, const int dims[4], int nc, dirac_prec prec, double rho,
                      int nsteps, void *stream);
/* Chain rule of a link derivative through stout smearing (the paper has no
 * force; derived here): with V = dirac_stout_smear(U, rho, nsteps) and G_V in
 * the convention of DIRAC_FORCE_GRAD (dS = Re sum conj(G_V) dV for any
 * complex dV, e.g. dirac_force of an operator built from V), G_U receives the
 * same for U: dS = Re sum conj(G_U) dU.  Per step V' = exp(iQ) U, in the form
 * dS = Re sum tr[dV' Sigma'] (Sigma' = G^dag):
 *   Sigma_U = Sigma' e^{iQ} - C^dag Xi + the staple terms of Y = U^dag Xi,
 *   Xi = anti-hermitian part of Lambda - tr(Lambda)/N_c,
 *   Lambda = L(iQ, U Sigma') the Frechet derivative of exp at iQ (computed
 *            as the upper-right block of exp([[iQ, U Sigma'], [0, iQ]])),
 * and each link of the staples in C_mu(x) receives rho times the derivative of
 * tr[(staple) Y_mu(x)] with respect to it.  U_in, G_V, G_U: device fields
 * [site][mu][a][b] complex in prec (F64 or F32), no boundary phases; G_U must
 * not alias U_in or G_V; N_c 1..4.  Arithmetic in FP64; the intermediate fields of the
 * forward steps are recomputed (nsteps - 1 fields plus three FP64 fields are
 * allocated and freed here).  Synchronises `stream`. */
int dirac_stout_backward(const void *U_in, const void *G_V, void *G_U, const int dims[4], int nc, dirac_prec prec,
                         double rho, int nsteps, void *stream);

/* Copy the operator's W links W_s(n) (Brillouin only) into the device
 * buffer w_out (w_bytes long, not overlapping the operator), layout
 * [site][80][a][b] (SITE_OUTER) or [80][a][b][site] (SITE_INNER) in the
 * link storage precision (geom->prec, FP32 with DIRAC_LINKS_F32),
 * directions s = (sx,sy,sz,st) in {-1,0,1}^4 numbered
 * d = (st+1)*27+(sz+1)*9+(sy+1)*3+(sx+1) with the centre d = 40 left out
 * (index d for d < 40, d-1 for d > 40).  Internally the operator stores
 * rho_k s_lead W_s, grouped by the axes s moves along; this call undoes the
 * order and the scale (one kernel on `stream`), so a 16-bit value can differ
 * from W_s rounded once by one more rounding.  Asynchronous on `stream`. */
int dirac_op_copy_w(const dirac_op *op, void *w_out, void *stream);

void dirac_op_destroy(dirac_op *op);

/* psi_out = D psi_in with bare mass m0 (Wilson Eq. app_wils, Brillouin
 * Eq. app_bril, staggered Eq. def_stag; plus the clover term when one is set,
 * dirac_op_set_clover).  psi_in and psi_out are vectors of the operator's
 * kind and precision and must not overlap. */
int dirac_apply(const dirac_op *op, const void *psi_in, void *psi_out, double m0, void *stream);

/* psi_out = D^dag psi_in: gamma5 D gamma5 for Wilson and Brillouin,
 * epsilon D epsilon for staggered (App. F, the forms the solvers use). */
int dirac_apply_dagger(const dirac_op *op, const void *psi_in, void *psi_out, double m0, void *stream);

/* psi_out = D^dag D psi_in (App. F, app_*dag*), through an operator-owned
 * scratch vector: calls on one operator must not run concurrently. */
int dirac_apply_normal(const dirac_op *op, const void *psi_in, void *psi_out, double m0, void *stream);

/* End-to-end apply from HOST memory: copies host_in to an operator-owned
 * device buffer, applies D (dagger != 0: D^dag), copies the result to
 * host_out and synchronises `stream`.  Host buffers of vec_bytes each;
 * pinned memory gives full copy bandwidth.  For N_t >= 3 the work runs in up
 * to 8 slabs of whole time slices: copies in on one operator-owned stream,
 * the stencil on `stream` for each slab whose t-neighbour slabs have
 * arrived, copies out on another operator-owned stream, all overlapping.
 * Calls on one operator must not run concurrently. */
int dirac_apply_host(const dirac_op *op, const void *host_in, void *host_out, double m0,
                     int dagger, void *stream);
/* dirac_apply_host without the final synchronisation, so that the host
 * applies of several operators overlap (one operator's stencil runs while
 * another's slabs are copied).  Returns once everything is enqueued; host_out
 * is complete when `stream` reaches the point after the call.  The copies
 * and the stencils run on operator-owned streams and wait only for this
 * operator's previous host apply (its staging buffers), not for earlier work
 * on `stream`, so host_in must be ready when the call is made.  Both host
 * buffers must stay valid (and host_in unchanged) until then; calls on one
 * operator are ordered, calls on different operators may share `stream`. */
int dirac_apply_host_async(const dirac_op *op, const void *host_in, void *host_out, double m0,
                           int dagger, void *stream);

/* ------------------------------------------------- domain decomposition
 * A lattice split into slabs of time slices, one per GPU (the paper leaves
 * distributed memory to future work, Sec. 1; App. A notes that the spin
 * projection halves a Wilson halo).  A slab operator is an ordinary operator
 * whose t extent is N_t,local + 2: slices 0 and N_t,local + 1 are ghost copies
 * of the neighbouring slabs' edge slices, links included (the caller folds the
 * global boundary phase into its links and passes bc[3] = +1).  Each stencil
 * reaches one slice in t, so these two ghost slices are the whole halo.
 *
 * dirac_apply_range: D (dagger = 0) or D^dag psi for the output sites
 * [site0, site0 + nsites) only (site order of the layout; the owned slices of
 * a slab operator are site0 = N_x N_y N_z, nsites = N_t,local N_x N_y N_z);
 * other output sites are left untouched.  Asynchronous on `stream`.
 *
 * dirac_halo_pack / dirac_halo_unpack: copy time slice t of a vector into a
 * contiguous buffer and back.  proj = 0: the full slice, order
 * [site in slice][colour][spin][v]; proj = a = +-1 (Wilson-type vectors only):
 * the half spinor h = upper two spin components of (1 + a gamma_4) psi
 * (gamma_4 of App. A), unpacked as (1 + a gamma_4) psi / 2, whose
 * (1 + a gamma_4) projection is exactly (1 + a gamma_4) psi: the D_W hop into
 * a ghost slice then gives the full-spinor result with half the bytes.  D_W
 * applies (1 - gamma_4) to the slice above and (1 + gamma_4) to the slice
 * below (signs swapped for the dagger).  dirac_halo_bytes gives the buffer
 * size (0 for invalid arguments).  Asynchronous on `stream`. */
int dirac_apply_range(const dirac_op *op, const void *psi_in, void *psi_out, double m0, int dagger,
                      long long site0, long long nsites, void *stream);
size_t dirac_halo_bytes(const dirac_op *op, int proj);
int dirac_halo_pack(const dirac_op *op, const void *v, int t, int proj, void *buf, void *stream);
int dirac_halo_unpack(const dirac_op *op, const void *buf, int t, int proj, void *v, void *stream);

/* ----------------------------------------------------- launch tuning
 * A stencil launch variant is (vr, minb, block): vr = right-hand sides per
 * thread (1, 2 or 4, dividing N_v); minb = register class, the cap of minb
 * resident 128-thread blocks per SM (1 = the compiler's choice; 3, 4, 5, 6
 * compiled for N_c = 3 only); block = threads per block, a multiple of 32 up
 * to 128 minb (0 = 128).  vr = 0 restores the default choice.  Errors:
 * DIRAC_ERR_INVALID_ARG for a variant that is not compiled, a vr that does
 * not divide N_v or a block size out of range. */
int dirac_op_set_launch(dirac_op *op, int vr, int minb, int block);
int dirac_op_get_launch(const dirac_op *op, int *vr, int *minb, int *block);
/* Time every compiled variant of D (bare mass m0) on operator-owned buffers
 * and keep the fastest for this operator; the choice is also remembered for
 * operators created later in this process with the same kind, layout,
 * precision, link storage, N_c, N_v and volume (including the
 * lower-precision twins of mixed solves).
 * best_ms (may be NULL) receives the winner's time per apply.  Synchronises. */
int dirac_op_autotune(dirac_op *op, double m0, void *stream, double *best_ms);

/* Bytes of one vector of this operator (sites x internal dofs x N_v x complex). */
size_t dirac_vec_bytes(const dirac_op *op);

/* ---------------------------------------------------------- BLAS-1 (Sec. 3)
 * Per-RHS vector operations on vectors of the operator's shape and precision.
 * Reductions keep FP64-level accuracy (Sec. 3 accumulates sp norms in dp):
 * FP64 arithmetic for FP64 vectors; for FP32/16-bit vectors, exact products
 * and compensated sums in FP32 per thread, FP64 across threads.  The order is
 * fixed (two-pass reduction), so results are bitwise reproducible.
 * out/coefficient arrays are DEVICE arrays of N_v entries. */
int dirac_vec_norm2(const dirac_op *op, const void *v, double *out_dev, void *stream);
/* <u, v> per RHS, linear in the second argument; out_dev holds N_v (re, im) pairs. */
int dirac_vec_dot(const dirac_op *op, const void *u, const void *v, double *out_dev, void *stream);
/* y += alpha x per RHS (Eq. def_incr with complex alpha); alpha_dev: N_v (re, im) pairs. */
int dirac_vec_axpy(const dirac_op *op, const double *alpha_dev, const void *x, void *y, void *stream);
/* z = a x + b y per RHS; a_dev, b_dev: N_v (re, im) pairs; z may alias x or y. */
int dirac_vec_axpby(const dirac_op *op, const double *a_dev, const void *x, const double *b_dev, const void *y,
                    void *z, void *stream);
/* dirac_vec_norm2 / dirac_vec_dot over the sites [site0, site0 + nsites)
 * only (site order of the layout; 1 <= nsites, site0 + nsites <= volume,
 * else DIRAC_ERR_INVALID_ARG): the owned sites of a slab operator, whose
 * ghost slices must not enter the dot products of a distributed solver. */
int dirac_vec_norm2_range(const dirac_op *op, const void *v, long long site0, long long nsites, double *out_dev,
                          void *stream);
int dirac_vec_dot_range(const dirac_op *op, const void *u, const void *v, long long site0, long long nsites,
                        double *out_dev, void *stream);
/* v = gamma5 v (4 spin components) or epsilon v (colour-only vectors), in place. */
int dirac_vec_gamma5(const dirac_op *op, void *v, void *stream);
/* Convert a vector between precisions (same shape): src in src_prec, dst in dst_prec. */
int dirac_vec_convert(const dirac_op *op, const void *src, dirac_prec src_prec, void *dst,
                      dirac_prec dst_prec, void *stream);

/* Per-RHS squared 2-norms of a [rows][nv] complex vector in precision prec,
 * written to out_dev (nv doubles), for callers that cannot allocate device
 * memory: code whose device memory is all owned by a pooling or caching
 * allocator that must not be bypassed, latency-critical loops that cannot
 * afford the implicit device synchronisation cudaMalloc/cudaFree may cause,
 * and programs running so close to the memory limit that a late allocation
 * could fail mid-solve.  It needs no operator handle and allocates nothing:
 * the partial sums live in a fixed device array inside the library
 * (DIRAC_NOALLOC_MAX_BLOCKS x 64 doubles = 256 KiB, held by every GPU that
 * loads the library until the process exits).  The paper has no counterpart;
 * the result equals dirac_vec_norm2's up to FP64 rounding (the two may split
 * the sum over a different number of blocks).
 *   v        device pointer, 16-byte aligned, rows*nv complex numbers
 *   rows     >= 1 (any size; the reduction is a grid-stride loop)
 *   nv       1..64: nv < 1 gives DIRAC_ERR_INVALID_ARG, nv > 64 DIRAC_ERR_CAPACITY
 * The first call on each device looks up the array's device address (with
 * that device current), so make that first call before any stream capture.
 * All calls share the one array: calls whose work overlaps on the GPU (other
 * streams, other host threads) race and must be serialised by the caller.
 * Nothing needs clearing between calls: every partial sum read is written
 * earlier in the same call. */
#define DIRAC_NOALLOC_MAX_BLOCKS 512
int dirac_vec_norm2_noalloc(const void *v, dirac_prec prec, long long rows, int nv, double *out_dev,
                            void *stream);

/* ------------------------------------------------------------- solvers (Sec. 9) */
typedef enum {
    DIRAC_CG_NORMAL = 0,   /* CG on D^dag D x = D^dag b (Sec. 9, A = D^dag D) */
    DIRAC_BICGSTAB = 1,    /* BiCGstab on D x = b (Sec. 9) */
    DIRAC_CG_HPD = 2       /* CG on D^dag D x = b, b given directly (pseudofermion solves);
                              for the Laplace kinds CG on A x = b with A itself (the
                              paper's cg_wlap / cg_blap), the only CG they accept */
} dirac_solver;

typedef struct {
    dirac_solver solver;   /* CG on D^dag D x = D^dag b, or BiCGstab on D x = b */
    double tol;            /* relative residual: ||r_N||/||D^dag b|| (CG) or ||b-Dx||/||b|| */
    int maxit;             /* total iteration limit (inner iterations for mixed solves) */
    dirac_prec inner_prec; /* == op precision: plain Krylov solve in that precision;
                              lower precision: mixed-precision solve (Sec. 9 "mp"
                              solvers) with residual, norms, convergence test and
                              solution in the operator's precision and the Krylov
                              iterations in inner_prec */
    double inner_tol;      /* restarted mode: relative tolerance of each inner solve (0 = default) */
    int recompute_every;   /* 0 = paper default: 50 for F64 solves, 20 otherwise */
    int mixed_mode;        /* DIRAC_MIXED_RELIABLE (CG only), DIRAC_MIXED_RESTART or
                              DIRAC_MIXED_ADAPTIVE (CG only) */
    int sloppy_links;      /* link storage of the inner operator: DIRAC_LINKS_NATIVE or
                              DIRAC_LINKS_F32 (16-bit inner vectors with FP32 links) */
    double delta;          /* reliable updates: recompute when the sloppy residual fell by
                              this factor since the last update (0 = default 0.1) */
} dirac_solve_params;

/* Mixed-precision strategies.  RESTART: defect correction, the paper's "mp"
 * driver (Sec. 9): r = b - A x in the operator precision, an inner solve of
 * A e = r/|r| from zero in inner_prec, x += |r| e, repeat.  RELIABLE (CG):
 * one Krylov iteration in inner_prec on the scaled residual, with the
 * solution and the true residual refreshed in the operator precision each
 * time the iterated residual has dropped by delta; the search direction is
 * kept across refreshes.  ADAPTIVE (CG, 16-bit inner_prec, FP64 operator):
 * RELIABLE in inner_prec while the refreshes keep halving the true residual
 * (2 refreshes in a row that fail to end it), then RELIABLE with an FP32
 * iteration from the current solution, within the same maxit; the stats
 * count both phases (no counterpart in the paper).  For other inner
 * precisions it is RELIABLE.  BiCGstab always uses RESTART. */
enum { DIRAC_MIXED_RELIABLE = 0, DIRAC_MIXED_RESTART = 1, DIRAC_MIXED_ADAPTIVE = 2 };

typedef struct {
    int iters;                 /* Krylov iterations (summed over inner solves) */
    int outer_iters;           /* defect-correction steps (0 for a plain solve) */
    int recomputes;            /* explicit residual recomputations */
    int status;                /* overall outcome: 0 or a positive code above */
    int status_per_rhs[64];
    double relres[64];         /* final recomputed residual, per RHS */
    double true_relres[64];    /* ||b - D x|| / ||b|| per RHS */
    double seconds;            /* wall time of the call */
    double lambda_min[64];     /* CG only: Lanczos estimates of the extreme eigenvalues */
    double lambda_max[64];     /* of D^dag D from the CG coefficients (App. F "cond"); 0 otherwise */
    int host_launches;         /* dirac_solve_batched: graph launches issued by the host (1 when the
                                  whole convergence loop ran as one graph with a device-side loop) */
    int iters_16bit;           /* RELIABLE / ADAPTIVE CG with a 16-bit inner_prec: iterations run
                                  with 16-bit sloppy vectors (ADAPTIVE: before the FP32 hand-over) */
    double seconds_16bit;      /* wall time of those iterations, refreshes included */
} dirac_solve_stats;

/* Solve for N_v right-hand sides b (operator precision); x holds the initial
 * guess on entry and the solution on exit.  Blocks until done (it reads
 * per-iteration residual norms on the host).  stats may be NULL. */
int dirac_solve(const dirac_op *op, const void *b, void *x, double m0,
                const dirac_solve_params *params, dirac_solve_stats *stats, void *stream);

/* Many independent solves at once (the paper's solvers, Sec. 9, grown into a
 * batch): solve i is CG on D_i^dag D_i x_i = D_i^dag b_i (DIRAC_CG_NORMAL) or
 * D_i^dag D_i x_i = b_i (DIRAC_CG_HPD) with operator ops[i] (distinct
 * handles: each solve uses its operator's workspace; any lattice, N_v and
 * kind), mass m0[i] (host array) and the shared tolerance and iteration
 * limit of params (inner_prec must equal every operator's precision).
 * Coefficients and convergence masks stay on the device; segments of
 * recompute_every (default 20) iterations followed by a true-residual
 * recompute run for all solves inside one CUDA graph whose device-side while
 * node repeats them (each solve behind its own conditional node, skipped once
 * converged) until every solve has converged or maxit is reached: one graph
 * launch by the host (a host replay of a one-segment graph where conditional
 * nodes are unavailable).  stats (host array of nsolves, may be NULL) receive per-solve
 * iterations (segment granularity), final residuals and the device-timed
 * seconds from the batch start to that solve's completion.  Blocks until done.
 * Returns 0 when all converged, DIRAC_NOT_CONVERGED otherwise. */
int dirac_solve_batched(int nsolves, dirac_op *const *ops, const void *const *b, void *const *x,
                        const double *m0, const dirac_solve_params *params, dirac_solve_stats *stats,
                        void *stream);

/* ------------------------------------------------------------ fermion force
 * Derivative of S = sum_v Re phi_v^dag (D^dag D)^-1 phi_v with respect to
 * the links, for D = D_W (Eq. app_wils), D_S (Eq. def_stag) or D_B (Eq.
 * app_bril, through the path-averaged W links of Tab. off-axis) (the paper
 * has no force; derived here, without the clover term, so an operator
 * carrying one is refused).  Inputs: psi = (D^dag D)^-1 phi and chi = D psi,
 * vectors of op (F64 or F32).  Output: [site][mu][a][b] complex in op precision.
 *   mode DIRAC_FORCE_TA:   F_mu(n) = P_TA(U B - C U^dag), traceless
 *                          anti-hermitian, with dS/deps = Re sum tr[X F] for
 *                          U -> exp(eps X) U, X in su(Nc);
 *   mode DIRAC_FORCE_GRAD: G with dS = Re sum conj(G) dU for an arbitrary
 *                          complex change dU of the caller's (unphased) links,
 * where, summed over spin and RHS,
 *   D_W: B_mu(n) = sum psi(n+mu) [(1-gamma_mu) chi(n)]^dag,
 *        C_mu(n) = sum psi(n) [(1+gamma_mu) chi(n+mu)]^dag;
 *   D_S: B_mu(n) = -eta_mu(n) sum psi(n+mu) chi(n)^dag,
 *        C_mu(n) =  eta_mu(n) sum psi(n) chi(n+mu)^dag;
 *   D_B: B_mu(n) = K_mu(n), C = 0, with dS = Re sum tr[dU K] from
 *        M_s(n) = sum (S_s psi(n+s)) chi(n)^dag, S_s = rho_k sum s_mu gamma_mu
 *        - lambda_k/2, carried back through the level recursion of W_s.
 *        The Brillouin force keeps a scratch of 216 N_c x N_c matrices per
 *        site in the handle (allocated on the first call, freed with it). */
enum { DIRAC_FORCE_TA = 0, DIRAC_FORCE_GRAD = 1 };
int dirac_force(const dirac_op *op, const void *psi, const void *chi, void *force_out, int mode, void *stream);
/* dirac_force restricted to D_W (DIRAC_ERR_INVALID_ARG for other kinds). */
int dirac_force_wilson(const dirac_op *op, const void *psi, const void *chi, void *force_out, int mode,
                       void *stream);

/* ------------------------------------------------------------- utilities */
const char *dirac_error_string(int code);
/* Flops per site per RHS (App. E): Wilson 128Nc^2+72Nc, Brillouin
 * 2560Nc^2+2376Nc, staggered 64Nc^2+2Nc; Laplace operators: WLAP
 * 256Nc^2+8Nc, BLAP 2560Nc^2+648Nc, WSUV 64Nc^2+2Nc, BSUV 640Nc^2+162Nc;
 * -1 for an invalid kind. */
long dirac_flops_per_site(dirac_kind kind, int nc);
/* Flops per site per RHS of the clover term as App. E counts it for the
 * two-multiplication form: 64Nc^2 (576 for SU(3)). */
long dirac_clover_flops_per_site(int nc);
/* Measured FP32 FMA peak of the current device, the denominator of the ALU
 * roofline the Brillouin stencil (App. E: 30168 flop per site and RHS for
 * SU(3), about 45 flop per algorithmic byte at N_v = 12) is reported against.
 * Runs an FMA-only kernel (8 independent chains per thread, 8 x 256 threads per
 * SM, `iters` x 128 FMAs per chain) once untimed and once timed with CUDA
 * events on `stream`; *tflops receives 2 x FMAs / time in TFLOP/s and
 * *sm_count (may be NULL) the device's multiprocessor count.  Synchronises
 * `stream`.  iters < 1 or tflops == NULL: DIRAC_ERR_INVALID_ARG. */
int dirac_measure_fp32_peak(int iters, double *tflops, int *sm_count, void *stream);
/* Compile-time library version (major*10000 + minor*100 + patch). */
int dirac_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DIRAC_H */
