// blas.cu -- multi-RHS linear algebra of Sec. 3 on the RHS-innermost layout:
// a vector is a [rows][nv] array of complex numbers (rows = sites x internal
// dofs), and every operation acts column by column with its own coefficient.
//
// Reductions (norm^2, dot) carry at least FP64-like precision whatever the
// storage precision (Sec. 3 accumulates sp norms in dp) and are
// deterministic: a fixed grid of blocks, thread (r, v) of a block owns column
// v, partial sums are combined in a fixed tree inside the block and then
// summed in block order by a second one-block kernel.  FP64 vectors
// accumulate in FP64.  FP32 and 16-bit vectors accumulate per thread in FP32
// with error-free transformations (Dekker's product, Knuth's two-sum): every
// product is split exactly into a rounded part and its error, the rounded
// parts are summed with their rounding errors collected, and the pair
// (sum, error) goes to the FP64 block reduction.  That keeps the thread
// loops on the FP32 pipe: FP64 arithmetic on this GPU runs at a small
// fraction of the FP32 rate and would limit the reductions far below HBM
// bandwidth.
//
// Every thread handles four rows per loop trip so that four independent
// 16-byte loads per operand are in flight.
#include <atomic>

#include "internal.h"

namespace dgb {

constexpr int kRedThreads = 256;

// Complex numbers per thread and per access: one 16-byte load when N_v allows.
inline int blas_group(dirac_prec p, int nv) { return pick_vr(p, nv); }

// Threads per block: a multiple of the number of column groups nv/G.
inline int red_block(int ngroups) { return ngroups * (kRedThreads / ngroups); }

// Reduce the per-thread column sums vals[G][NOUT] over the R row-threads of the
// block (fixed pairwise tree) and store the block's partial sums for its nv
// columns: partial_block[v][NOUT].
template <int G, int NOUT>
__device__ __forceinline__ void block_reduce_store(const double (&vals)[G][NOUT], double *sh, int r, int vg, int R,
                                                   int ng, double *partial_block) {
    constexpr int W = G * NOUT;
#pragma unroll
    for (int i = 0; i < G; ++i)
#pragma unroll
        for (int q = 0; q < NOUT; ++q) sh[(r * ng + vg) * W + i * NOUT + q] = vals[i][q];
    __syncthreads();
    for (int off = 1; off < R; off *= 2) {
        if ((r % (2 * off)) == 0 && r + off < R) {
#pragma unroll
            for (int w = 0; w < W; ++w) sh[(r * ng + vg) * W + w] += sh[((r + off) * ng + vg) * W + w];
        }
        __syncthreads();
    }
    if (r == 0) {
#pragma unroll
        for (int i = 0; i < G; ++i)
#pragma unroll
            for (int q = 0; q < NOUT; ++q) partial_block[(vg * G + i) * NOUT + q] = sh[vg * W + i * NOUT + q];
    }
}

// Second pass of a reduction: partial[b][col] (col = v*NOUT + q, cols =
// nv*NOUT) -> out[col].  One block of kFinThreads threads: T = kFinThreads /
// cols threads per column each sum the blocks t, t+T, ... in order, then a
// fixed pairwise tree combines the T partial sums, so the result does not
// depend on timing.  KEEP = 1 keeps only q = 0 of each v (the real part of a
// dot product) and writes out[v].
constexpr int kFinThreads = 256;
template <int NOUT, int KEEP>
__global__ void __launch_bounds__(kFinThreads) finalize_kernel(const double *__restrict__ partial, int nblocks,
                                                               int nv, double *__restrict__ out) {
    __shared__ double sh[kFinThreads];
    const int cols = nv * KEEP;
    const int T = kFinThreads / cols;
    const int t = threadIdx.x / cols, c = threadIdx.x % cols;
    // column c of the output is column src of the partials
    const int src = KEEP == NOUT ? c : c * NOUT;
    double acc = 0.0;
    if (t < T)
        for (int b = t; b < nblocks; b += T) acc += partial[(long long)b * nv * NOUT + src];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int off = 1; off < T; off *= 2) {
        if (t % (2 * off) == 0 && t + off < T) sh[t * cols + c] += sh[(t + off) * cols + c];
        __syncthreads();
    }
    if (t == 0) out[c] = sh[c];
}

// Per-thread accumulator of a real sum.  FP64 data: a plain double.  FP32
// data: (s, c) with the exact value s + c of everything added so far up to
// the errors of the error-free steps (Knuth's two-sum and Dekker's product via
// FMA); the explicit __f*_rn intrinsics keep the compiler from contracting or
// reassociating them.
template <typename A>
struct RedAcc;
template <>
struct RedAcc<double> {
    double s = 0.0;
    __device__ __forceinline__ void mac(double x, double y) { s = fma(x, y, s); }
    __device__ __forceinline__ double value() const { return s; }
};
template <>
struct RedAcc<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float p) {
        const float t = __fadd_rn(s, p);
        const float bp = __fsub_rn(t, s);
        c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp)));
        s = t;
    }
    __device__ __forceinline__ void mac(float x, float y) {
        const float p = __fmul_rn(x, y);
        add(p);
        c = __fadd_rn(c, __fmaf_rn(x, y, -p));
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// thread (r, vg) of a block walks the rows r0 = block*R + r, stride grid*R and
// owns columns vg*G .. vg*G+G-1
#define BLAS_THREAD_SETUP                                   \
    const int ng = nv / G;                                  \
    const int R = blockDim.x / ng;                          \
    const int r = threadIdx.x / ng, vg = threadIdx.x % ng;  \
    const bool live = r < R;                                \
    const long long stride = (long long)gridDim.x * R;

// Rows of a reduction over part of a vector: `rows` logical rows in segments
// of seg_len, segment k starting at row k * seg_stride + seg_off (the sites
// [site0, site0 + nsites) of every component of a site-inner vector).
struct RowMap {
    long long seg_len = 0, seg_stride = 0, seg_off = 0;   // seg_len = 0: identity
    __device__ __forceinline__ long long operator()(long long row) const {
        return seg_len ? (row / seg_len) * seg_stride + seg_off + row % seg_len : row;
    }
};

template <typename E, int G>
__global__ void norm2_kernel(const E *__restrict__ x, long long rows, int nv, double *__restrict__ partial,
                             RowMap rm = RowMap{}) {
    extern __shared__ double sh[];
    using A = typename Acc<E>::T;
    BLAS_THREAD_SETUP
    RedAcc<A> acc[G];
    auto add = [&](const cx<A> (&a)[G]) {
#pragma unroll
        for (int i = 0; i < G; ++i) {
            acc[i].mac(a[i].re, a[i].re);
            acc[i].mac(a[i].im, a[i].im);
        }
    };
    if (live) {
        long long row = (long long)blockIdx.x * R + r;
        for (; row + 3 * stride < rows; row += 4 * stride) {
            cx<A> a[4][G];
#pragma unroll
            for (int u = 0; u < 4; ++u) load_cx<E, G, A>(x + 2 * (rm(row + u * stride) * nv + vg * G), a[u]);
#pragma unroll
            for (int u = 0; u < 4; ++u) add(a[u]);
        }
        for (; row < rows; row += stride) {
            cx<A> a[1][G];
            load_cx<E, G, A>(x + 2 * (rm(row) * nv + vg * G), a[0]);
            add(a[0]);
        }
    }
    double out[G][1];
#pragma unroll
    for (int i = 0; i < G; ++i) out[i][0] = acc[i].value();
    block_reduce_store<G, 1>(out, sh, r, vg, R, ng, partial + (long long)blockIdx.x * nv);
}

template <typename E, int G>
__global__ void dot_kernel(const E *__restrict__ x, const E *__restrict__ y, long long rows, int nv,
                           double *__restrict__ partial, RowMap rm = RowMap{}) {
    extern __shared__ double sh[];
    using A = typename Acc<E>::T;
    BLAS_THREAD_SETUP
    RedAcc<A> re[G], im[G];
    auto add = [&](const cx<A> (&a)[G], const cx<A> (&b)[G]) {
#pragma unroll
        for (int i = 0; i < G; ++i) {   // conj(x) * y
            re[i].mac(a[i].re, b[i].re);
            re[i].mac(a[i].im, b[i].im);
            im[i].mac(a[i].re, b[i].im);
            im[i].mac(-a[i].im, b[i].re);
        }
    };
    if (live) {
        long long row = (long long)blockIdx.x * R + r;
        for (; row + 3 * stride < rows; row += 4 * stride) {
            cx<A> a[4][G], b[4][G];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const long long e = 2 * (rm(row + u * stride) * nv + vg * G);
                load_cx<E, G, A>(x + e, a[u]);
                load_cx<E, G, A>(y + e, b[u]);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) add(a[u], b[u]);
        }
        for (; row < rows; row += stride) {
            cx<A> a[1][G], b[1][G];
            const long long e = 2 * (rm(row) * nv + vg * G);
            load_cx<E, G, A>(x + e, a[0]);
            load_cx<E, G, A>(y + e, b[0]);
            add(a[0], b[0]);
        }
    }
    double out[G][2];
#pragma unroll
    for (int i = 0; i < G; ++i) {
        out[i][0] = re[i].value();
        out[i][1] = im[i].value();
    }
    block_reduce_store<G, 2>(out, sh, r, vg, R, ng, partial + 2LL * blockIdx.x * nv);
}

template <typename A>
__device__ __forceinline__ cx<A> coef(const double *c, double scale, int v) {
    return c ? cx<A>{(A)(scale * c[2 * v]), (A)(scale * c[2 * v + 1])} : cx<A>{(A)scale, (A)0};
}

// z = a x + b y per column; a, b = scale * coef[v] (complex pairs) or scale
// alone when coef is null; x or y may be null (term dropped); z may alias x
// or y.  With partial != null also reduces |z|^2 per column.
template <typename E, int G>
__global__ void axpby_kernel(E *z, const E *x, const E *y, const double *__restrict__ ac, double as,
                             const double *__restrict__ bc, double bs, long long rows, int nv, double *partial) {
    extern __shared__ double sh[];
    using A = typename Acc<E>::T;
    BLAS_THREAD_SETUP
    cx<A> a[G], b[G];
#pragma unroll
    for (int i = 0; i < G; ++i) {
        a[i] = coef<A>(ac, as, vg * G + i);
        b[i] = coef<A>(bc, bs, vg * G + i);
    }
    RedAcc<A> acc[G];
    // one row: combine, store, and (optionally) add |z|^2 of the value as
    // stored: the registers rounded through the storage type (z may alias x
    // or y, so it is not re-read)
    auto finish = [&](long long e, const cx<A> (&tx)[G], const cx<A> (&ty)[G]) {
        cx<A> out[G];
#pragma unroll
        for (int i = 0; i < G; ++i) {
            out[i] = cx<A>{0, 0};
            if (x) cmac(out[i], a[i], tx[i]);
            if (y) cmac(out[i], b[i], ty[i]);
        }
        store_cx<E, G, A>(z + e, out);
        if (partial) {
#pragma unroll
            for (int i = 0; i < G; ++i) {
                const A re = (A)to_acc<E>(from_acc<E, A>(out[i].re));
                const A im = (A)to_acc<E>(from_acc<E, A>(out[i].im));
                acc[i].mac(re, re);
                acc[i].mac(im, im);
            }
        }
    };
    if (live) {
        long long row = (long long)blockIdx.x * R + r;
        for (; row + 3 * stride < rows; row += 4 * stride) {
            cx<A> tx[4][G], ty[4][G];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const long long e = 2 * ((row + u * stride) * nv + vg * G);
                if (x) load_cx<E, G, A>(x + e, tx[u]);
                if (y) load_cx<E, G, A>(y + e, ty[u]);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) finish(2 * ((row + u * stride) * nv + vg * G), tx[u], ty[u]);
        }
        for (; row < rows; row += stride) {
            const long long e = 2 * (row * nv + vg * G);
            cx<A> tx[1][G], ty[1][G];
            if (x) load_cx<E, G, A>(x + e, tx[0]);
            if (y) load_cx<E, G, A>(y + e, ty[0]);
            finish(e, tx[0], ty[0]);
        }
    }
    if (partial) {
        double out[G][1];
#pragma unroll
        for (int i = 0; i < G; ++i) out[i][0] = acc[i].value();
        block_reduce_store<G, 1>(out, sh, r, vg, R, ng, partial + (long long)blockIdx.x * nv);
    }
}

// The two Krylov updates that use the old search direction, in one pass:
// x += a p, then p = r + b p.
template <typename E, int G>
__global__ void update_xp_kernel(E *x, E *p, const E *__restrict__ r_, const double *__restrict__ ac,
                                 const double *__restrict__ bc, long long rows, int nv) {
    using A = typename Acc<E>::T;
    BLAS_THREAD_SETUP
    if (!live) return;
    cx<A> a[G], b[G];
#pragma unroll
    for (int i = 0; i < G; ++i) {
        a[i] = coef<A>(ac, 1.0, vg * G + i);
        b[i] = coef<A>(bc, 1.0, vg * G + i);
    }
    auto finish = [&](long long e, cx<A> (&xv)[G], cx<A> (&pv)[G], const cx<A> (&rv)[G]) {
#pragma unroll
        for (int i = 0; i < G; ++i) {
            cmac(xv[i], a[i], pv[i]);
            cx<A> np = rv[i];
            cmac(np, b[i], pv[i]);
            pv[i] = np;
        }
        store_cx<E, G, A>(x + e, xv);
        store_cx<E, G, A>(p + e, pv);
    };
    long long row = (long long)blockIdx.x * R + r;
    for (; row + 3 * stride < rows; row += 4 * stride) {
        cx<A> xv[4][G], pv[4][G], rv[4][G];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const long long e = 2 * ((row + u * stride) * nv + vg * G);
            load_cx<E, G, A>(x + e, xv[u]);
            load_cx<E, G, A>(p + e, pv[u]);
            load_cx<E, G, A>(r_ + e, rv[u]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) finish(2 * ((row + u * stride) * nv + vg * G), xv[u], pv[u], rv[u]);
    }
    for (; row < rows; row += stride) {
        const long long e = 2 * (row * nv + vg * G);
        cx<A> xv[1][G], pv[1][G], rv[1][G];
        load_cx<E, G, A>(x + e, xv[0]);
        load_cx<E, G, A>(p + e, pv[0]);
        load_cx<E, G, A>(r_ + e, rv[0]);
        finish(e, xv[0], pv[0], rv[0]);
    }
}

#undef BLAS_THREAD_SETUP

template <typename F>
static int dispatch_group(int g, F &&f) {
    switch (g) {
    case 1: return f(std::integral_constant<int, 1>{});
    case 2: return f(std::integral_constant<int, 2>{});
    case 4: return f(std::integral_constant<int, 4>{});
    }
    return DIRAC_ERR_INVALID_ARG;
}

// launch geometry shared by the reduction kernels: threads per block, shared bytes
struct RedLaunch {
    int G, tb;
    size_t sh;
};
static RedLaunch red_launch(dirac_prec p, int nv, int nout) {
    RedLaunch L;
    L.G = blas_group(p, nv);
    const int ng = nv / L.G;
    L.tb = red_block(ng);
    // one extra row of slots absorbs the threads beyond R (tb is a multiple of ng)
    L.sh = (size_t)(L.tb + ng) * L.G * nout * sizeof(double);
    return L;
}

template <typename E>
__global__ void gamma5_kernel(E *__restrict__ v, Lat g, int nc, int staggered, int layout) {
    const long long rows = staggered ? g.V * nc : g.V * nc * 4;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * g.nv) return;
    const long long row = i / g.nv;   // (site, cs) site-outer or (cs, site) site-inner
    bool neg;
    if (staggered) {
        const Coord c = site_coords(g, layout == 0 ? row / nc : row % g.V);
        neg = (c.x + c.y + c.z + c.t) & 1;        // epsilon(n) = (-1)^(x+y+z+t)
    } else {
        const long long spin = layout == 0 ? row % 4 : (row / g.V) % 4;
        neg = spin >= 2;                          // gamma5 = diag(1, 1, -1, -1)
    }
    if (neg) {
        using A = typename Acc<E>::T;
        v[2 * i] = from_acc<E, A>(-to_acc<E>(v[2 * i]));
        v[2 * i + 1] = from_acc<E, A>(-to_acc<E>(v[2 * i + 1]));
    }
}

template <typename S, typename D>
__global__ void convert_kernel(const S *__restrict__ src, D *__restrict__ dst, long long count) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) dst[i] = from_acc<D, typename Acc<S>::T>(to_acc<S>(src[i]));
}

// Deterministic pseudo-random fill in [-1, 1) (a 32-bit integer hash of the
// element index), used to give timing runs realistic, non-zero operands.
template <typename E>
__global__ void fill_hash_kernel(E *__restrict__ v, long long count, unsigned seed) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    unsigned h = (unsigned)i * 2654435761u ^ seed;
    h ^= h >> 16;
    h *= 2246822519u;
    h ^= h >> 13;
    h *= 3266489917u;
    h ^= h >> 16;
    const float f = (float)(h >> 8) * (1.0f / 8388608.0f) - 1.0f;
    v[i] = from_acc<E, typename Acc<E>::T>((typename Acc<E>::T)f);
}

int blas_fill_hash(const dirac_op *op, dirac_prec p, void *v, unsigned seed, cudaStream_t s) {
    return dispatch_prec(p, [&](auto tag) {
        using E = std::remove_pointer_t<decltype(tag)>;
        const long long n = op->rows * op->nv * 2;
        fill_hash_kernel<E><<<grid_for(n, 256), 256, 0, s>>>((E *)v, n, seed);
        return launch_check("fill_hash_kernel");
    });
}

static inline int red_grid(const dirac_op *op) { return op->red_blocks; }

template <typename E>
static int launch_norm2(const E *v, long long rows, int nv, dirac_prec p, double *partial, int blocks, double *out,
                        cudaStream_t s) {
    const RedLaunch L = red_launch(p, nv, 1);
    return dispatch_group(L.G, [&](auto gc) {
        constexpr int G = decltype(gc)::value;
        norm2_kernel<E, G><<<blocks, L.tb, L.sh, s>>>(v, rows, nv, partial);
        finalize_kernel<1, 1><<<1, kFinThreads, 0, s>>>(partial, blocks, nv, out);
        return launch_check("norm2_kernel");
    });
}

int blas_norm2(const dirac_op *op, dirac_prec p, const void *v, double *out, cudaStream_t s) {
    return dispatch_prec(p, [&](auto tag) {
        using E = std::remove_pointer_t<decltype(tag)>;
        return launch_norm2<E>((const E *)v, op->rows, op->nv, p, op->red_partial, red_grid(op), out, s);
    });
}

int blas_dot(const dirac_op *op, dirac_prec p, const void *u, const void *v, double *out, cudaStream_t s) {
    return dispatch_prec(p, [&](auto tag) {
        using E = std::remove_pointer_t<decltype(tag)>;
        const RedLaunch L = red_launch(p, op->nv, 2);
        return dispatch_group(L.G, [&](auto gc) {
            constexpr int G = decltype(gc)::value;
            dot_kernel<E, G><<<red_grid(op), L.tb, L.sh, s>>>((const E *)u, (const E *)v, op->rows, op->nv,
                                                              op->red_partial);
            finalize_kernel<2, 2><<<1, kFinThreads, 0, s>>>(op->red_partial, red_grid(op), op->nv, out);
            return launch_check("dot_kernel");
        });
    });
}

int blas_dot_re(const dirac_op *op, dirac_prec p, const void *u, const void *v, double *out, cudaStream_t s) {
    return dispatch_prec(p, [&](auto tag) {
        using E = std::remove_pointer_t<decltype(tag)>;
        const RedLaunch L = red_launch(p, op->nv, 2);
        return dispatch_group(L.G, [&](auto gc) {
            constexpr int G = decltype(gc)::value;
            dot_kernel<E, G><<<red_grid(op), L.tb, L.sh, s>>>((const E *)u, (const E *)v, op->rows, op->nv,
                                                              op->red_partial);
            finalize_kernel<2, 1><<<1, kFinThreads, 0, s>>>(op->red_partial, red_grid(op), op->nv, out);
            return launch_check("dot_kernel");
        });
    });
}

// The rows of sites [site0, site0 + nsites): one run for site-outer vectors,
// one run per internal component for site-inner ones.
static void site_rows(const dirac_op *op, long long site0, long long nsites, long long &first, long long &rows,
                      RowMap &rm) {
    const long long ncs = op->rows / op->V;
    rows = nsites * ncs;
    if (op->geom.layout == DIRAC_LAYOUT_SITE_OUTER) {
        first = site0 * ncs;
        rm = RowMap{};
    } else {
        first = 0;
        rm = RowMap{nsites, op->V, site0};
    }
}

int blas_norm2_range(const dirac_op *op, dirac_prec p, const void *v, long long site0, long long nsites, double *out,
                     cudaStream_t s) {
    long long first, rows;
    RowMap rm;
    site_rows(op, site0, nsites, first, rows, rm);
    return dispatch_prec(p, [&](auto tag) {
        using E = std::remove_pointer_t<decltype(tag)>;
        const RedLaunch L = red_launch(p, op->nv, 1);
        return dispatch_group(L.G, [&](auto gc) {
            constexpr int G = decltype(gc)::value;
            norm2_kernel<E, G><<<red_grid(op), L.tb, L.sh, s>>>((const E *)v + 2 * first * op->nv, rows, op->nv,
                                                                op->red_partial, rm);
            finalize_kernel<1, 1><<<1, kFinThreads, 0, s>>>(op->red_partial, red_grid(op), op->nv, out);
            return launch_check("norm2_kernel");
        });
    });
}

int blas_dot_range(const dirac_op *op, dirac_prec p, const void *u, const void *v, long long site0, long long nsites,
                   double *out, cudaStream_t s) {
    long long first, rows;
    RowMap rm;
    site_rows(op, site0, nsites, first, rows, rm);
    return dispatch_prec(p, [&](auto tag) {
        using E = std::remove_pointer_t<decltype(tag)>;
        const RedLaunch L = red_launch(p, op->nv, 2);
        return dispatch_group(L.G, [&](auto gc) {
            constexpr int G = decltype(gc)::value;
            dot_kernel<E, G><<<red_grid(op), L.tb, L.sh, s>>>((const E *)u + 2 * first * op->nv,
                                                              (const E *)v + 2 * first * op->nv, rows, op->nv,
                                                              op->red_partial, rm);
            finalize_kernel<2, 2><<<1, kFinThreads, 0, s>>>(op->red_partial, red_grid(op), op->nv, out);
            return launch_check("dot_kernel");
        });
    });
}

int blas_axpby(const dirac_op *op, dirac_prec p, void *z, const void *x, const double *a, double as, const void *y,
               const double *b, double bs, double *norm_out, cudaStream_t s) {
    return dispatch_prec(p, [&](auto tag) {
        using E = std::remove_pointer_t<decltype(tag)>;
        const RedLaunch L = red_launch(p, op->nv, 1);
        return dispatch_group(L.G, [&](auto gc) {
            constexpr int G = decltype(gc)::value;
            axpby_kernel<E, G><<<red_grid(op), L.tb, L.sh, s>>>((E *)z, (const E *)x, (const E *)y, a, as, b, bs,
                                                                op->rows, op->nv,
                                                                norm_out ? op->red_partial : nullptr);
            if (norm_out) finalize_kernel<1, 1><<<1, kFinThreads, 0, s>>>(op->red_partial, red_grid(op), op->nv, norm_out);
            return launch_check("axpby_kernel");
        });
    });
}

int blas_axpy(const dirac_op *op, dirac_prec p, const double *alpha, const void *x, void *y, cudaStream_t s) {
    return blas_axpby(op, p, y, x, alpha, 1.0, y, nullptr, 1.0, nullptr, s);
}

int blas_update_xp(const dirac_op *op, dirac_prec p, void *x, void *pv, const void *r, const double *a,
                   const double *b, cudaStream_t s) {
    return dispatch_prec(p, [&](auto tag) {
        using E = std::remove_pointer_t<decltype(tag)>;
        const RedLaunch L = red_launch(p, op->nv, 1);
        return dispatch_group(L.G, [&](auto gc) {
            constexpr int G = decltype(gc)::value;
            update_xp_kernel<E, G><<<red_grid(op), L.tb, 0, s>>>((E *)x, (E *)pv, (const E *)r, a, b, op->rows,
                                                                 op->nv);
            return launch_check("update_xp_kernel");
        });
    });
}

int blas_gamma5(const dirac_op *op, dirac_prec p, void *v, cudaStream_t s) {
    return dispatch_prec(p, [&](auto tag) {
        using E = std::remove_pointer_t<decltype(tag)>;
        const long long n = op->rows * op->nv;
        gamma5_kernel<E><<<grid_for(n, 256), 256, 0, s>>>((E *)v, op->lat, op->nc, spins_of(op->kind) == 1,
                                                          op->geom.layout);
        return launch_check("gamma5_kernel");
    });
}

int blas_convert(const dirac_op *op, const void *src, dirac_prec sp, void *dst, dirac_prec dp, cudaStream_t s) {
    return dispatch_prec(sp, [&](auto stag) {
        using S = std::remove_pointer_t<decltype(stag)>;
        return dispatch_prec(dp, [&](auto dtag) {
            using D = std::remove_pointer_t<decltype(dtag)>;
            const long long n = op->rows * op->nv * 2;
            convert_kernel<S, D><<<grid_for(n, 256), 256, 0, s>>>((const S *)src, (D *)dst, n);
            return launch_check("convert_kernel");
        });
    });
}

// ------------------------------------------------------------------------
// Allocation-free variant of the norm^2 reduction (dirac_vec_norm2_noalloc):
// the per-block partial sums go to a file-scope device array instead of the
// operator's buffer.  Host code must not pass the symbol itself to a kernel
// (in host code it names a host-side shadow, not device memory): its device
// address is looked up once per device with cudaGetSymbolAddress.
static __device__ __align__(256) double g_noalloc_partial[DIRAC_NOALLOC_MAX_BLOCKS * 64];

static double *noalloc_partial_ptr(int *rc) {
    // one cached device address per device; host threads may race on the
    // first lookup, so the slots are atomics (every racer stores the same value)
    static std::atomic<double *> addr[128];
    int dev = 0;
    *rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
    if (*rc) return nullptr;
    if (dev < 0 || dev >= 128) {
        *rc = DIRAC_ERR_CAPACITY;
        return nullptr;
    }
    double *p = addr[dev].load(std::memory_order_acquire);
    if (!p) {
        *rc = cuda_check(cudaGetSymbolAddress((void **)&p, g_noalloc_partial), "cudaGetSymbolAddress");
        if (*rc) return nullptr;
        addr[dev].store(p, std::memory_order_release);
    }
    return p;
}

}  // namespace dgb

extern "C" int dirac_vec_norm2_noalloc(const void *v, dirac_prec prec, long long rows, int nv, double *out_dev,
                                       void *stream) {
    using namespace dgb;
    if (!v || !out_dev || rows < 1) return DIRAC_ERR_INVALID_ARG;
    if ((uintptr_t)v & 15) return DIRAC_ERR_ALIGNMENT;
    if (prec < DIRAC_F64 || prec > DIRAC_F16) return DIRAC_ERR_UNSUPPORTED_PREC;
    if (nv < 1) return DIRAC_ERR_INVALID_ARG;
    if (nv > 64) {
        fprintf(stderr, "libdirac: dirac_vec_norm2_noalloc: nv = %d exceeds the static capacity of 64\n", nv);
        return DIRAC_ERR_CAPACITY;
    }
    int rc = DIRAC_OK;
    double *partial = noalloc_partial_ptr(&rc);
    if (rc) return rc;
    const RedLaunch L = red_launch(prec, nv, 1);
    const int R = L.tb / (nv / L.G);
    long long want = (rows + R - 1) / R;
    const int blocks = (int)(want < DIRAC_NOALLOC_MAX_BLOCKS ? want : DIRAC_NOALLOC_MAX_BLOCKS);
    cudaStream_t s = (cudaStream_t)stream;
    return dispatch_prec(prec, [&](auto tag) {
        using E = std::remove_pointer_t<decltype(tag)>;
        return launch_norm2<E>((const E *)v, rows, nv, prec, partial, blocks, out_dev, s);
    });
}
