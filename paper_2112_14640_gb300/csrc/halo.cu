// halo.cu -- the time-slice halos of a lattice split into slabs along t
// (one slab per GPU; the paper leaves MPI to future work, Sec. 1, and App. A
// notes that the spin projection halves what a Wilson halo has to carry).
//
// A slab operator is an ordinary operator on N_t,local + 2 time slices: the
// first and the last slice are ghost copies of the neighbouring slabs' edge
// slices, and only the owned slices 1..N_t,local are computed
// (dirac_apply_range).  Every stencil here reaches one slice in t, so one
// ghost slice on each side is the whole halo, for D_W, D_S and D_B alike.
//
// Pack / unpack move one time slice (all sites of slice t, every colour,
// spin and RHS) between a vector and a contiguous buffer:
//   proj = 0:       the full slice (any kind);
//   proj = a = +-1: Wilson-type vectors only, the half spinor
//                   h = the upper two spin components of (1 + a gamma_4) psi
//                   (in the chiral basis of App. A (1 + a gamma_4) psi =
//                   (psi0 + a psi2, psi1 + a psi3, a h0, a h1)); unpacking
//                   writes (1 + a gamma_4) psi / 2 = (h0, h1, a h0, a h1) / 2,
//                   whose (1 + a gamma_4) projection is exactly (1 + a gamma_4) psi,
//                   so a stencil hop that applies that projector to the ghost
//                   gets the same value as from the full spinor, with half
//                   the bytes on the wire.  The forward t-hop of D_W applies
//                   (1 - sgn gamma_4) to the slice above, the backward hop
//                   (1 + sgn gamma_4) to the slice below (sgn = -1: dagger).
#include "internal.h"

namespace dgb {

// buffer order: [site in slice][colour][spin (4, or 2 for half spinors, or 1)][v]
template <typename E, int LAYOUT>
__global__ void halo_pack_kernel(const E *__restrict__ v, E *__restrict__ buf, Lat g, int ncs, int nc, int ns, int t,
                                 int proj) {
    const long long slice = (long long)g.nx * g.ny * g.nz;
    const int nso = proj ? 2 : ns;   // spin components per colour in the buffer
    const long long total = slice * nc * nso * g.nv;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int vv = (int)(i % g.nv);
    long long r = i / g.nv;
    const int s = (int)(r % nso);
    r /= nso;
    const int c = (int)(r % nc);
    const long long site = (long long)t * slice + r / nc;
    using L = Layout<LAYOUT>;
    const long long cs = L::cs_stride(g);
    const long long base = L::vec(g, site, ncs, 0) + vv;
    using A = typename Acc<E>::T;
    if (!proj) {
        const long long o = base + (long long)(c * ns + s) * cs;
        buf[2 * i] = v[2 * o];
        buf[2 * i + 1] = v[2 * o + 1];
        return;
    }
    // h_s = psi_s + a psi_{s+2}, s = 0, 1
    const long long o0 = base + (long long)(c * 4 + s) * cs, o2 = base + (long long)(c * 4 + s + 2) * cs;
    const A a = (A)proj;
    buf[2 * i] = from_acc<E, A>(to_acc<E>(v[2 * o0]) + a * to_acc<E>(v[2 * o2]));
    buf[2 * i + 1] = from_acc<E, A>(to_acc<E>(v[2 * o0 + 1]) + a * to_acc<E>(v[2 * o2 + 1]));
}

template <typename E, int LAYOUT>
__global__ void halo_unpack_kernel(const E *__restrict__ buf, E *__restrict__ v, Lat g, int ncs, int nc, int ns, int t,
                                   int proj) {
    const long long slice = (long long)g.nx * g.ny * g.nz;
    const int nso = proj ? 2 : ns;
    const long long total = slice * nc * nso * g.nv;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int vv = (int)(i % g.nv);
    long long r = i / g.nv;
    const int s = (int)(r % nso);
    r /= nso;
    const int c = (int)(r % nc);
    const long long site = (long long)t * slice + r / nc;
    using L = Layout<LAYOUT>;
    const long long cs = L::cs_stride(g);
    const long long base = L::vec(g, site, ncs, 0) + vv;
    using A = typename Acc<E>::T;
    if (!proj) {
        const long long o = base + (long long)(c * ns + s) * cs;
        v[2 * o] = buf[2 * i];
        v[2 * o + 1] = buf[2 * i + 1];
        return;
    }
    // (h0, h1, a h0, a h1) / 2
    const A a = (A)proj, hre = (A)0.5 * to_acc<E>(buf[2 * i]), him = (A)0.5 * to_acc<E>(buf[2 * i + 1]);
    const long long o0 = base + (long long)(c * 4 + s) * cs, o2 = base + (long long)(c * 4 + s + 2) * cs;
    v[2 * o0] = from_acc<E, A>(hre);
    v[2 * o0 + 1] = from_acc<E, A>(him);
    v[2 * o2] = from_acc<E, A>(a * hre);
    v[2 * o2 + 1] = from_acc<E, A>(a * him);
}

static int halo_check(const dirac_op *op, int t, int proj) {
    if (!op || t < 0 || t >= op->lat.nt || proj < -1 || proj > 1) return DIRAC_ERR_INVALID_ARG;
    if (proj && spins_of(op->kind) != 4) return DIRAC_ERR_INVALID_ARG;   // half spinors: Wilson-type vectors only
    return DIRAC_OK;
}

size_t halo_elems(const dirac_op *op, int proj) {
    const long long slice = (long long)op->lat.nx * op->lat.ny * op->lat.nz;
    const int nso = proj ? 2 : spins_of(op->kind);
    return (size_t)slice * op->nc * nso * op->nv;   // complex numbers
}

template <bool PACK>
static int halo_move(const dirac_op *op, const void *src, void *dst, int t, int proj, cudaStream_t s) {
    int rc = halo_check(op, t, proj);
    if (rc) return rc;
    const long long total = (long long)halo_elems(op, proj);
    const int ns = spins_of(op->kind), ncs = op->nc * ns;
    return dispatch_prec(op->prec, [&](auto tag) {
        using E = std::remove_pointer_t<decltype(tag)>;
        return dispatch_layout(op->geom.layout, [&](auto lyc) {
            constexpr int LAYOUT = decltype(lyc)::value;
            if (PACK)
                halo_pack_kernel<E, LAYOUT><<<grid_for(total, 256), 256, 0, s>>>((const E *)src, (E *)dst, op->lat, ncs,
                                                                                 op->nc, ns, t, proj);
            else
                halo_unpack_kernel<E, LAYOUT><<<grid_for(total, 256), 256, 0, s>>>((const E *)src, (E *)dst, op->lat,
                                                                                   ncs, op->nc, ns, t, proj);
            return launch_check(PACK ? "halo_pack_kernel" : "halo_unpack_kernel");
        });
    });
}

}  // namespace dgb

using namespace dgb;

extern "C" size_t dirac_halo_bytes(const dirac_op *op, int proj) {
    if (!op || proj < -1 || proj > 1 || (proj && spins_of(op->kind) != 4)) return 0;
    return halo_elems(op, proj) * 2 * elem_bytes(op->prec);
}

extern "C" int dirac_halo_pack(const dirac_op *op, const void *v, int t, int proj, void *buf, void *stream) {
    if (!v || !buf) return DIRAC_ERR_INVALID_ARG;
    return halo_move<true>(op, v, buf, t, proj, (cudaStream_t)stream);
}

extern "C" int dirac_halo_unpack(const dirac_op *op, const void *buf, int t, int proj, void *v, void *stream) {
    if (!v || !buf) return DIRAC_ERR_INVALID_ARG;
    return halo_move<false>(op, buf, v, t, proj, (cudaStream_t)stream);
}

extern "C" int dirac_apply_range(const dirac_op *op, const void *psi_in, void *psi_out, double m0, int dagger,
                                 long long site0, long long nsites, void *stream) {
    if (!op || !psi_in || !psi_out || psi_in == psi_out) return DIRAC_ERR_INVALID_ARG;
    if (((uintptr_t)psi_in & 15) || ((uintptr_t)psi_out & 15)) return DIRAC_ERR_ALIGNMENT;
    if (site0 < 0 || nsites < 0 || site0 + nsites > op->V) return DIRAC_ERR_INVALID_ARG;
    if (nsites == 0) return DIRAC_OK;
    dirac_op part = *op;   // same buffers, output sites [site0, site0 + nsites) only
    part.lat.n0 = site0;
    part.lat.nsites = nsites;
    return op_apply(&part, psi_in, psi_out, m0, dagger ? -1 : +1, (cudaStream_t)stream);
}
