// blas.cu -- multi-RHS linear algebra of Sec. 3 on the RHS-innermost layout:
// a vector is a [rows][nv] array of complex numbers (rows = sites x internal
// dofs), and every operation acts column by column with its own coefficient.
//
// Reductions (norm^2, dot) accumulate in FP64 whatever the storage precision
// (Sec. 3 accumulates sp norms in dp) and are deterministic: a fixed grid of
// blocks, thread (r, v) of a block owns column v, partial sums are combined in
// a fixed tree inside the block and then summed in block order by a second
// one-block kernel.
#include "internal.h"

namespace dgb {

constexpr int kRedThreads = 256;

// threads per block that are a multiple of nv (one column per thread)
inline int red_block(int nv) { return nv * (kRedThreads / nv); }

template <int NOUT>
__device__ __forceinline__ void block_reduce_store(double (*vals)[NOUT], double *sh, int r, int v, int R, int nv,
                                                   double *partial_block) {
    // sh holds R*nv*NOUT doubles
#pragma unroll
    for (int q = 0; q < NOUT; ++q) sh[(r * nv + v) * NOUT + q] = (*vals)[q];
    __syncthreads();
    for (int off = 1; off < R; off *= 2) {
        if ((r % (2 * off)) == 0 && r + off < R) {
#pragma unroll
            for (int q = 0; q < NOUT; ++q) sh[(r * nv + v) * NOUT + q] += sh[((r + off) * nv + v) * NOUT + q];
        }
        __syncthreads();
    }
    if (r == 0) {
#pragma unroll
        for (int q = 0; q < NOUT; ++q) partial_block[v * NOUT + q] = sh[v * NOUT + q];
    }
}

// partial[b][v][NOUT] -> out[v][NOUT], summed in block order
template <int NOUT>
__global__ void finalize_kernel(const double *__restrict__ partial, int nblocks, int nv, double *__restrict__ out) {
    const int v = threadIdx.x;
    if (v >= nv) return;
    double acc[NOUT];
#pragma unroll
    for (int q = 0; q < NOUT; ++q) acc[q] = 0.0;
    for (int b = 0; b < nblocks; ++b)
#pragma unroll
        for (int q = 0; q < NOUT; ++q) acc[q] += partial[((long long)b * nv + v) * NOUT + q];
#pragma unroll
    for (int q = 0; q < NOUT; ++q) out[v * NOUT + q] = acc[q];
}

template <typename E>
__global__ void norm2_kernel(const E *__restrict__ x, long long rows, int nv, double *__restrict__ partial) {
    extern __shared__ double sh[];
    const int R = blockDim.x / nv;
    const int r = threadIdx.x / nv, v = threadIdx.x % nv;
    double acc[1] = {0.0};
    for (long long row = (long long)blockIdx.x * R + r; row < rows; row += (long long)gridDim.x * R) {
        const long long e = 2 * (row * nv + v);
        const double re = (double)to_acc<E>(x[e]), im = (double)to_acc<E>(x[e + 1]);
        acc[0] = fma(re, re, acc[0]);
        acc[0] = fma(im, im, acc[0]);
    }
    block_reduce_store<1>(&acc, sh, r, v, R, nv, partial + (long long)blockIdx.x * nv);
}

template <typename E>
__global__ void dot_kernel(const E *__restrict__ x, const E *__restrict__ y, long long rows, int nv,
                           double *__restrict__ partial) {
    extern __shared__ double sh[];
    const int R = blockDim.x / nv;
    const int r = threadIdx.x / nv, v = threadIdx.x % nv;
    double acc[2] = {0.0, 0.0};
    for (long long row = (long long)blockIdx.x * R + r; row < rows; row += (long long)gridDim.x * R) {
        const long long e = 2 * (row * nv + v);
        const double xr = (double)to_acc<E>(x[e]), xi = (double)to_acc<E>(x[e + 1]);
        const double yr = (double)to_acc<E>(y[e]), yi = (double)to_acc<E>(y[e + 1]);
        // conj(x) * y
        acc[0] = fma(xr, yr, acc[0]);
        acc[0] = fma(xi, yi, acc[0]);
        acc[1] = fma(xr, yi, acc[1]);
        acc[1] = fma(-xi, yr, acc[1]);
    }
    block_reduce_store<2>(&acc, sh, r, v, R, nv, partial + 2LL * blockIdx.x * nv);
}

// z = a x + b y per column; a, b = scale * coef[v] (complex pairs) or scale
// alone when coef is null; x or y may be null (term dropped); z may alias x
// or y.  With partial != null also reduces |z|^2 per column.
template <typename E>
__global__ void axpby_kernel(E *z, const E *x, const E *y, const double *__restrict__ ac, double as,
                             const double *__restrict__ bc, double bs, long long rows, int nv, double *partial) {
    extern __shared__ double sh[];
    using A = typename Acc<E>::T;
    const int R = blockDim.x / nv;
    const int r = threadIdx.x / nv, v = threadIdx.x % nv;
    const double ar = ac ? as * ac[2 * v] : as, ai = ac ? as * ac[2 * v + 1] : 0.0;
    const double br = bc ? bs * bc[2 * v] : bs, bi = bc ? bs * bc[2 * v + 1] : 0.0;
    const cx<A> a = {(A)ar, (A)ai}, b = {(A)br, (A)bi};
    double acc[1] = {0.0};
    for (long long row = (long long)blockIdx.x * R + r; row < rows; row += (long long)gridDim.x * R) {
        const long long e = 2 * (row * nv + v);
        cx<A> out = {0, 0};
        if (x) cmac(out, a, cx<A>{(A)to_acc<E>(x[e]), (A)to_acc<E>(x[e + 1])});
        if (y) cmac(out, b, cx<A>{(A)to_acc<E>(y[e]), (A)to_acc<E>(y[e + 1])});
        const E zr = from_acc<E, A>(out.re), zi = from_acc<E, A>(out.im);
        z[e] = zr;
        z[e + 1] = zi;
        if (partial) {
            const double dr = (double)to_acc<E>(zr), di = (double)to_acc<E>(zi);
            acc[0] = fma(dr, dr, acc[0]);
            acc[0] = fma(di, di, acc[0]);
        }
    }
    if (partial) block_reduce_store<1>(&acc, sh, r, v, R, nv, partial + (long long)blockIdx.x * nv);
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

int blas_norm2(const dirac_op *op, dirac_prec p, const void *v, double *out, cudaStream_t s) {
    return dispatch_prec(p, [&](auto tag) {
        using E = std::remove_pointer_t<decltype(tag)>;
        const int tb = red_block(op->nv);
        norm2_kernel<E><<<red_grid(op), tb, tb * sizeof(double), s>>>((const E *)v, op->rows, op->nv, op->red_partial);
        finalize_kernel<1><<<1, 64, 0, s>>>(op->red_partial, red_grid(op), op->nv, out);
        return launch_check("norm2_kernel");
    });
}

int blas_dot(const dirac_op *op, dirac_prec p, const void *u, const void *v, double *out, cudaStream_t s) {
    return dispatch_prec(p, [&](auto tag) {
        using E = std::remove_pointer_t<decltype(tag)>;
        const int tb = red_block(op->nv);
        dot_kernel<E><<<red_grid(op), tb, 2 * tb * sizeof(double), s>>>((const E *)u, (const E *)v, op->rows, op->nv,
                                                                       op->red_partial);
        finalize_kernel<2><<<1, 64, 0, s>>>(op->red_partial, red_grid(op), op->nv, out);
        return launch_check("dot_kernel");
    });
}

int blas_axpby(const dirac_op *op, dirac_prec p, void *z, const void *x, const double *a, double as, const void *y,
               const double *b, double bs, double *norm_out, cudaStream_t s) {
    return dispatch_prec(p, [&](auto tag) {
        using E = std::remove_pointer_t<decltype(tag)>;
        const int tb = red_block(op->nv);
        axpby_kernel<E><<<red_grid(op), tb, tb * sizeof(double), s>>>(
            (E *)z, (const E *)x, (const E *)y, a, as, b, bs, op->rows, op->nv, norm_out ? op->red_partial : nullptr);
        if (norm_out) finalize_kernel<1><<<1, 64, 0, s>>>(op->red_partial, red_grid(op), op->nv, norm_out);
        return launch_check("axpby_kernel");
    });
}

int blas_axpy(const dirac_op *op, dirac_prec p, const double *alpha, const void *x, void *y, cudaStream_t s) {
    return blas_axpby(op, p, y, x, alpha, 1.0, y, nullptr, 1.0, nullptr, s);
}

int blas_gamma5(const dirac_op *op, dirac_prec p, void *v, cudaStream_t s) {
    return dispatch_prec(p, [&](auto tag) {
        using E = std::remove_pointer_t<decltype(tag)>;
        const long long n = op->rows * op->nv;
        gamma5_kernel<E><<<grid_for(n, 256), 256, 0, s>>>((E *)v, op->lat, op->nc, op->kind == DIRAC_STAGGERED,
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
    static double *addr[128] = {nullptr};
    int dev = 0;
    *rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
    if (*rc) return nullptr;
    if (dev < 0 || dev >= 128) {
        *rc = DIRAC_ERR_CAPACITY;
        return nullptr;
    }
    if (!addr[dev]) {
        double *p = nullptr;
        *rc = cuda_check(cudaGetSymbolAddress((void **)&p, g_noalloc_partial), "cudaGetSymbolAddress");
        if (*rc) return nullptr;
        addr[dev] = p;
    }
    return addr[dev];
}

}  // namespace dgb

extern "C" int dirac_vec_norm2_noalloc(const void *v, dirac_prec prec, long long rows, int nv, double *out_dev,
                                       void *stream) {
    using namespace dgb;
    if (!v || !out_dev || rows < 1) return DIRAC_ERR_INVALID_ARG;
    if ((uintptr_t)v & 15) return DIRAC_ERR_ALIGNMENT;
    if (prec < DIRAC_F64 || prec > DIRAC_F16) return DIRAC_ERR_UNSUPPORTED_PREC;
    if (nv < 1 || nv > 64) {
        fprintf(stderr, "libdirac: dirac_vec_norm2_noalloc: nv = %d exceeds the static capacity of 64\n", nv);
        return DIRAC_ERR_CAPACITY;
    }
    int rc = DIRAC_OK;
    double *partial = noalloc_partial_ptr(&rc);
    if (rc) return rc;
    const int tb = red_block(nv);
    const int R = tb / nv;
    long long want = (rows + R - 1) / R;
    const int blocks = (int)(want < DIRAC_NOALLOC_MAX_BLOCKS ? want : DIRAC_NOALLOC_MAX_BLOCKS);
    cudaStream_t s = (cudaStream_t)stream;
    return dispatch_prec(prec, [&](auto tag) {
        using E = std::remove_pointer_t<decltype(tag)>;
        norm2_kernel<E><<<blocks, tb, tb * sizeof(double), s>>>((const E *)v, rows, nv, partial);
        finalize_kernel<1><<<1, 64, 0, s>>>(partial, blocks, nv, out_dev);
        return launch_check("norm2_kernel (noalloc)");
    });
}
