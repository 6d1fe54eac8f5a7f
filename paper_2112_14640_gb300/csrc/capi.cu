// capi.cu -- the extern "C" entry points of include/dirac.h: argument
// validation, the operator handle (owned link/W copies, scratch and staging
// buffers, reduction partials), dispatch by operator kind, and error strings.
#include <stdlib.h>
#include <string.h>

#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "internal.h"

// Streams and events of the pipelined host apply (dirac_apply_host), which
// works in at most kMaxSlabs slabs of time slices.  Each operator has its own
// copy streams: the host applies of several operators enqueued back to back
// then copy concurrently, which measured faster than one copy-in stream shared
// by all of them in call order (16^3x32, N_v = 12, D_B + D_W + D_S: 2.74 vs
// 2.99 ms per step).
constexpr int kMaxSlabs = 8;
struct dirac_host_pipe {
    cudaStream_t h2d = nullptr, d2h = nullptr, comp = nullptr;   // comp: stencils of the asynchronous form
    cudaEvent_t in_done[kMaxSlabs] = {}, out_ready[kMaxSlabs] = {}, start = nullptr, end = nullptr;
    bool used = false;   // `end` has been recorded by an earlier call
};

using namespace dgb;

namespace dgb {

#define CTRY(x)                 \
    do {                        \
        int rc_ = (x);          \
        if (rc_) return rc_;    \
    } while (0)

int op_apply(const dirac_op *op, const void *in, void *out, double m0, int sgn, cudaStream_t s) {
    switch (op->kind) {
    case DIRAC_WILSON: return launch_wilson(op, in, out, m0, sgn, s);
    case DIRAC_BRILLOUIN: return launch_brillouin(op, in, out, m0, sgn, s);
    case DIRAC_STAGGERED: return launch_staggered(op, in, out, m0, sgn, s);
    case DIRAC_WLAP:
    case DIRAC_BLAP:
    case DIRAC_WSUV:
    case DIRAC_BSUV: return launch_laplace(op, in, out, m0, s);   // hermitian: sgn is irrelevant
    }
    return DIRAC_ERR_INVALID_ARG;
}

// D^dag D psi through the operator's scratch vector.
int op_apply_normal(const dirac_op *op, const void *in, void *out, double m0, cudaStream_t s) {
    int rc = op_apply(op, in, op->scratch, m0, +1, s);
    if (rc) return rc;
    return op_apply(op, op->scratch, out, m0, -1, s);
}

int op_apply_cg(const dirac_op *op, const void *in, void *out, double m0, cudaStream_t s) {
    return is_laplace(op->kind) ? op_apply(op, in, out, m0, +1, s) : op_apply_normal(op, in, out, m0, s);
}

static void pipe_free(dirac_host_pipe *p) {
    if (!p) return;
    for (int k = 0; k < kMaxSlabs; ++k) {
        if (p->in_done[k]) cudaEventDestroy(p->in_done[k]);
        if (p->out_ready[k]) cudaEventDestroy(p->out_ready[k]);
    }
    if (p->start) cudaEventDestroy(p->start);
    if (p->end) cudaEventDestroy(p->end);
    if (p->h2d) cudaStreamDestroy(p->h2d);
    if (p->d2h) cudaStreamDestroy(p->d2h);
    if (p->comp) cudaStreamDestroy(p->comp);
    delete p;
}

static int pipe_get(dirac_op *op, dirac_host_pipe **out) {
    if (!op->pipe) {
        dirac_host_pipe *p = new dirac_host_pipe();
        int rc = cuda_check(cudaStreamCreateWithFlags(&p->h2d, cudaStreamNonBlocking), "pipe stream");
        if (!rc) rc = cuda_check(cudaStreamCreateWithFlags(&p->d2h, cudaStreamNonBlocking), "pipe stream");
        if (!rc) rc = cuda_check(cudaStreamCreateWithFlags(&p->comp, cudaStreamNonBlocking), "pipe stream");
        for (int k = 0; k < kMaxSlabs && !rc; ++k) {
            rc = cuda_check(cudaEventCreateWithFlags(&p->in_done[k], cudaEventDisableTiming), "pipe event");
            if (!rc) rc = cuda_check(cudaEventCreateWithFlags(&p->out_ready[k], cudaEventDisableTiming), "pipe event");
        }
        if (!rc) rc = cuda_check(cudaEventCreateWithFlags(&p->start, cudaEventDisableTiming), "pipe event");
        if (!rc) rc = cuda_check(cudaEventCreateWithFlags(&p->end, cudaEventDisableTiming), "pipe event");
        if (rc) {
            pipe_free(p);
            return rc;
        }
        op->pipe = p;
    }
    *out = op->pipe;
    return DIRAC_OK;
}

static void op_free(dirac_op *op) {
    if (!op) return;
    pipe_free(op->pipe);
    for (int i = 0; i < 4; ++i)
        for (int k = 0; k < 2; ++k) op_free(op->inner[i][k]);
    cudaFree(op->links);
    cudaFree(op->w);
    cudaFree(op->clover);
    cudaFree(op->scratch);
    cudaFree(op->stage_in);
    cudaFree(op->stage_out);
    cudaFree(op->red_partial);
    cudaFree(op->solver_ws);
    cudaFree(op->force_ws);
    free(op);
}

static int validate_geom(dirac_kind kind, const dirac_geom *g) {
    if (!g) return DIRAC_ERR_INVALID_ARG;
    if (kind < DIRAC_WILSON || kind > DIRAC_BSUV) return DIRAC_ERR_INVALID_ARG;
    for (int m = 0; m < 4; ++m) {
        if (g->dims[m] < 2) return DIRAC_ERR_INVALID_ARG;
        if (g->bc[m] != 1 && g->bc[m] != -1) return DIRAC_ERR_INVALID_ARG;
        if (kind == DIRAC_STAGGERED && (g->dims[m] & 1)) return DIRAC_ERR_INVALID_ARG;
    }
    if ((long long)g->dims[0] * g->dims[1] * g->dims[2] * g->dims[3] > (1LL << 31)) return DIRAC_ERR_INVALID_ARG;
    if (g->prec < DIRAC_F64 || g->prec > DIRAC_F16) return DIRAC_ERR_UNSUPPORTED_PREC;
    // N_c 1..8 for FP64/FP32 vectors, 1..4 with 16-bit storage (internal.h)
    if (!nc_supported(g->nc, g->prec)) return DIRAC_ERR_UNSUPPORTED_NC;
    if (g->nv < 1 || g->nv > 64) return DIRAC_ERR_INVALID_ARG;
    if (g->layout != DIRAC_LAYOUT_SITE_OUTER && g->layout != DIRAC_LAYOUT_SITE_INNER) return DIRAC_ERR_INVALID_ARG;
    if (g->link_storage != DIRAC_LINKS_NATIVE && g->link_storage != DIRAC_LINKS_F32) return DIRAC_ERR_INVALID_ARG;
    if (g->link_storage == DIRAC_LINKS_F32 && g->prec != DIRAC_BF16 && g->prec != DIRAC_F16)
        return DIRAC_ERR_UNSUPPORTED_PREC;
    if (is_laplace(kind) && g->prec != DIRAC_F64 && g->prec != DIRAC_F32) return DIRAC_ERR_UNSUPPORTED_PREC;
    return DIRAC_OK;
}

static int alloc(void **p, size_t bytes) {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return DIRAC_ERR_OOM;
    }
    return DIRAC_OK;
}

// Process-wide memory of autotuned launch variants, keyed by what decides
// the kernel's behaviour.
// (kind, layout, precision, link storage, N_c, N_v, volume)
using TuneKey = std::tuple<int, int, int, int, int, int, long long, int>;
struct TuneVal {
    int vr, minb, block;
};
static std::mutex g_tune_mu;
static std::map<TuneKey, TuneVal> g_tune;

static TuneKey tune_key(const dirac_op *op) {
    return TuneKey{(int)op->kind, op->geom.layout, (int)op->prec, (int)link_prec(op), op->nc, op->nv, op->V,
                   op->clover != nullptr};
}

static void remember_tuning(const dirac_op *op) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[tune_key(op)] = TuneVal{op->vr, op->minb, op->block};
}

static void recall_tuning(dirac_op *op) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(tune_key(op));
    if (it != g_tune.end()) {
        op->vr = it->second.vr;
        op->minb = it->second.minb;
        op->block = it->second.block;
    }
}

// Allocate an operator handle of the given geometry without links.
int op_alloc(dirac_kind kind, const dirac_geom *g, dirac_op **out) {
    dirac_op *op = (dirac_op *)calloc(1, sizeof(dirac_op));
    if (!op) return DIRAC_ERR_OOM;
    op->kind = kind;
    op->geom = *g;
    op->nc = g->nc;
    op->nv = g->nv;
    op->prec = g->prec;
    op->V = (long long)g->dims[0] * g->dims[1] * g->dims[2] * g->dims[3];
    op->lat = Lat{g->dims[0], g->dims[1], g->dims[2], g->dims[3], g->nv, op->V, 0, op->V};
    op->rows = op->V * op->nc * spins_of(kind);
    const size_t eb = elem_bytes(op->prec), lb = elem_bytes(link_prec(op));
    op->vec_bytes = (size_t)op->rows * op->nv * 2 * eb;
    op->link_bytes = (size_t)link_sites(op->V) * 4 * op->nc * op->nc * 2 * lb;   // whole 32-site blocks
    op->w_bytes = uses_w(kind) ? (size_t)op->V * 80 * op->nc * op->nc * 2 * lb : 0;
    // one reduction block per 2 SMs' worth of work, at most 1216 blocks
    long long want = (op->rows + 255) / 256;
    op->red_blocks = (int)(want < 1216 ? (want < 1 ? 1 : want) : 1216);
    int rc = alloc(&op->links, op->link_bytes);
    if (!rc && op->w_bytes) rc = alloc(&op->w, op->w_bytes);
    if (!rc) rc = alloc(&op->scratch, op->vec_bytes);
    if (!rc) rc = alloc((void **)&op->red_partial, (size_t)op->red_blocks * op->nv * 2 * sizeof(double));
    if (rc) {
        op_free(op);
        return rc;
    }
    recall_tuning(op);
    *out = op;
    return DIRAC_OK;
}

// Lower-precision twin of op (same links/W converted), created once.
int op_inner(const dirac_op *op, dirac_prec p, int link_storage, dirac_op **out, cudaStream_t s) {
    if (p == op->prec) {
        *out = (dirac_op *)op;
        return DIRAC_OK;
    }
    if (p != DIRAC_BF16 && p != DIRAC_F16) link_storage = DIRAC_LINKS_NATIVE;
    dirac_op *self = (dirac_op *)op;
    if (!self->inner[p][link_storage]) {
        dirac_geom g = op->geom;
        g.prec = p;
        g.link_storage = link_storage;
        dirac_op *tw = nullptr;
        int rc = op_alloc(op->kind, &g, &tw);
        if (rc) return rc;
        if (op->clover) {
            tw->csw = op->csw;
            rc = alloc(&tw->clover, tw->link_bytes);
        }
        if (!rc) rc = launch_convert_links(op, tw, s);
        if (rc) {
            op_free(tw);
            return rc;
        }
        self->inner[p][link_storage] = tw;
    }
    *out = self->inner[p][link_storage];
    return DIRAC_OK;
}

void op_destroy(dirac_op *op) { op_free(op); }

}  // namespace dgb

static int check_vec(const void *p) {
    if (!p) return DIRAC_ERR_INVALID_ARG;
    if ((uintptr_t)p & 15) return DIRAC_ERR_ALIGNMENT;
    return DIRAC_OK;
}

// twins built from older links or another clover term are stale
static void drop_twins(dirac_op *op) {
    for (int i = 0; i < 4; ++i)
        for (int k = 0; k < 2; ++k) {
            op_destroy(op->inner[i][k]);
            op->inner[i][k] = nullptr;
        }
}

static int load_links(dirac_op *op, const void *U, dirac_prec u_prec, cudaStream_t s) {
    if (!U) return DIRAC_ERR_INVALID_ARG;
    if (u_prec != DIRAC_F64 && u_prec != DIRAC_F32) return DIRAC_ERR_UNSUPPORTED_PREC;
    int rc = launch_phase_links(op, U, u_prec, s);
    if (!rc && uses_w(op->kind)) rc = launch_build_w(op, U, u_prec, s);
    if (!rc) rc = cuda_check(cudaStreamSynchronize(s), "link setup");
    // a clover term belongs to the old field
    cudaFree(op->clover);
    op->clover = nullptr;
    op->csw = 0.0;
    drop_twins(op);
    return rc;
}

extern "C" {

int dirac_op_create(dirac_kind kind, const dirac_geom *geom, const void *U, dirac_prec u_prec, void *stream,
                    dirac_op **out) {
    if (!out) return DIRAC_ERR_INVALID_ARG;
    *out = nullptr;
    int rc = validate_geom(kind, geom);
    if (rc) return rc;
    if (!U) return DIRAC_ERR_INVALID_ARG;
    if (u_prec != DIRAC_F64 && u_prec != DIRAC_F32) return DIRAC_ERR_UNSUPPORTED_PREC;
    dirac_op *op = nullptr;
    rc = op_alloc(kind, geom, &op);
    if (rc) return rc;
    rc = load_links(op, U, u_prec, (cudaStream_t)stream);
    if (rc) {
        op_destroy(op);
        return rc;
    }
    *out = op;
    return DIRAC_OK;
}

int dirac_op_update_links(dirac_op *op, const void *U, dirac_prec u_prec, void *stream) {
    if (!op) return DIRAC_ERR_INVALID_ARG;
    return load_links(op, U, u_prec, (cudaStream_t)stream);
}

int dirac_op_set_clover(dirac_op *op, double csw, const void *V, dirac_prec v_prec, void *stream) {
    if (!op || (op->kind != DIRAC_WILSON && op->kind != DIRAC_BRILLOUIN) || !std::isfinite(csw))
        return DIRAC_ERR_INVALID_ARG;
    if (csw != 0.0) {
        if (!V) return DIRAC_ERR_INVALID_ARG;
        if (v_prec != DIRAC_F64 && v_prec != DIRAC_F32) return DIRAC_ERR_UNSUPPORTED_PREC;
    }
    cudaStream_t s = (cudaStream_t)stream;
    drop_twins(op);
    if (csw == 0.0) {
        int rc = op->clover ? cuda_check(cudaStreamSynchronize(s), "clover removal") : DIRAC_OK;
        cudaFree(op->clover);
        op->clover = nullptr;
        op->csw = 0.0;
        recall_tuning(op);
        return rc;
    }
    int rc = op->clover ? DIRAC_OK : alloc(&op->clover, op->link_bytes);
    if (rc) return rc;
    op->csw = csw;
    rc = launch_build_clover(op, V, v_prec, s);
    if (!rc) rc = cuda_check(cudaStreamSynchronize(s), "clover setup");
    if (rc) {
        cudaFree(op->clover);
        op->clover = nullptr;
        op->csw = 0.0;
    }
    recall_tuning(op);
    return rc;
}

int dirac_stout_smear(const void *U_in, void *V_out, const int dims[4], int nc, dirac_prec prec, double rho,
                      int nsteps, void *stream) {
    if (!U_in || !V_out || !dims || nsteps < 0 || nsteps > 1000 || !std::isfinite(rho)) return DIRAC_ERR_INVALID_ARG;
    for (int m = 0; m < 4; ++m)
        if (dims[m] < 2) return DIRAC_ERR_INVALID_ARG;
    if (prec != DIRAC_F64 && prec != DIRAC_F32) return DIRAC_ERR_UNSUPPORTED_PREC;
    if (!nc_supported(nc, prec)) return DIRAC_ERR_UNSUPPORTED_NC;
    const long long V = (long long)dims[0] * dims[1] * dims[2] * dims[3];
    if (V > (1LL << 31)) return DIRAC_ERR_INVALID_ARG;
    const size_t bytes = (size_t)V * 4 * nc * nc * 2 * elem_bytes(prec);
    cudaStream_t s = (cudaStream_t)stream;
    if (nsteps == 0)
        return U_in == V_out ? DIRAC_OK
                             : cuda_check(cudaMemcpyAsync(V_out, U_in, bytes, cudaMemcpyDeviceToDevice, s), "stout copy");
    const Lat g{dims[0], dims[1], dims[2], dims[3], 1, V, 0, V};
    void *tmp = nullptr;
    int rc = alloc(&tmp, bytes);
    if (rc) return rc;
    // steps alternate between V_out and tmp and never write the buffer they
    // read; an in-place call starts from a copy
    const void *src = U_in;
    if (U_in == V_out) {
        rc = cuda_check(cudaMemcpyAsync(tmp, U_in, bytes, cudaMemcpyDeviceToDevice, s), "stout copy");
        src = tmp;
    }
    for (int i = 0; i < nsteps && !rc; ++i) {
        void *dst = (src == V_out) ? tmp : V_out;
        rc = launch_stout_step(src, dst, g, nc, prec, rho, s);
        src = dst;
    }
    if (!rc && src != V_out)
        rc = cuda_check(cudaMemcpyAsync(V_out, src, bytes, cudaMemcpyDeviceToDevice, s), "stout copy");
    if (!rc) rc = cuda_check(cudaStreamSynchronize(s), "stout smear");
    cudaFree(tmp);
    return rc;
}

int dirac_stout_backward(const void *U_in, const void *G_V, void *G_U, const int dims[4], int nc, dirac_prec prec,
                         double rho, int nsteps, void *stream) {
    if (!U_in || !G_V || !G_U || !dims || nsteps < 0 || nsteps > 1000 || !std::isfinite(rho))
        return DIRAC_ERR_INVALID_ARG;
    for (int m = 0; m < 4; ++m)
        if (dims[m] < 2) return DIRAC_ERR_INVALID_ARG;
    if (prec != DIRAC_F64 && prec != DIRAC_F32) return DIRAC_ERR_UNSUPPORTED_PREC;
    if (!nc_supported(nc, prec)) return DIRAC_ERR_UNSUPPORTED_NC;
    const long long V = (long long)dims[0] * dims[1] * dims[2] * dims[3];
    if (V > (1LL << 31)) return DIRAC_ERR_INVALID_ARG;
    if (G_V == G_U || U_in == G_U) return DIRAC_ERR_INVALID_ARG;
    if (nc > kMaxNcSmall) return DIRAC_ERR_UNSUPPORTED_NC;
    const Lat g{dims[0], dims[1], dims[2], dims[3], 1, V, 0, V};
    return launch_stout_backward(U_in, G_V, G_U, g, nc, prec, rho, nsteps, (cudaStream_t)stream);
}

int dirac_op_copy_w(const dirac_op *op, void *w_out, void *stream) {
    if (!op || !w_out || !uses_w(op->kind)) return DIRAC_ERR_INVALID_ARG;
    return launch_unpack_w(op, w_out, (cudaStream_t)stream);
}

void dirac_op_destroy(dirac_op *op) { op_destroy(op); }

size_t dirac_vec_bytes(const dirac_op *op) { return op ? op->vec_bytes : 0; }

int dirac_op_set_launch(dirac_op *op, int vr, int minb, int block) {
    if (!op) return DIRAC_ERR_INVALID_ARG;
    if (vr == 0) {
        op->vr = op->minb = op->block = 0;
        return DIRAC_OK;
    }
    if (!variant_ok(op, vr, minb)) return DIRAC_ERR_INVALID_ARG;
    if (block == 0) block = kStencilBlock;
    if (block < 32 || block % 32 || block > stencil_max_threads(minb)) return DIRAC_ERR_INVALID_ARG;
    op->vr = vr;
    op->minb = minb;
    op->block = block;
    return DIRAC_OK;
}

int dirac_op_get_launch(const dirac_op *op, int *vr, int *minb, int *block) {
    if (!op || !vr || !minb || !block) return DIRAC_ERR_INVALID_ARG;
    launch_variant(op, *vr, *minb, *block);
    return DIRAC_OK;
}

int dirac_op_autotune(dirac_op *op, double m0, void *stream, double *best_ms) {
    if (!op) return DIRAC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = DIRAC_OK;
    if (!op->stage_out) rc = alloc(&op->stage_out, op->vec_bytes);
    if (rc) return rc;
    // realistic operands (power draw, and hence clocks, depend on the data)
    rc = blas_fill_hash(op, op->prec, op->scratch, 12345u, s);
    if (rc) return rc;
    struct Cand {
        int vr, minb, block;
        float ms;
    };
    std::vector<Cand> cands;
    const int vrs[3] = {1, 2, 4}, minbs[5] = {1, 3, 4, 5, 6}, blocks[5] = {128, 256, 384, 512, 768};
    for (int vr : vrs)
        for (int mb : minbs)
            for (int bl : blocks)
                if (variant_ok(op, vr, mb) && bl <= stencil_max_threads(mb))
                    cands.push_back(Cand{vr, mb, bl, 1e30f});
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int saved_vr = op->vr, saved_mb = op->minb, saved_bl = op->block;
    // three interleaved rounds, best time per variant, so that a clock or
    // neighbour transient does not decide the choice
    for (int round = 0; round < 3 && !rc; ++round)
        for (Cand &c : cands) {
            if (rc) break;
            op->vr = c.vr;
            op->minb = c.minb;
            op->block = c.block;
            rc = op_apply(op, op->scratch, op->stage_out, m0, +1, s);
            const int reps = 5;
            cudaEventRecord(e0, s);
            for (int r = 0; r < reps && !rc; ++r) rc = op_apply(op, op->scratch, op->stage_out, m0, +1, s);
            cudaEventRecord(e1, s);
            if (!rc) rc = cuda_check(cudaEventSynchronize(e1), "autotune sync");
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= reps;
            if (ms < c.ms) c.ms = ms;
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const Cand *best = nullptr;
    for (const Cand &c : cands)
        if (!best || c.ms < best->ms) best = &c;
    if (rc || !best) {
        op->vr = saved_vr;
        op->minb = saved_mb;
        op->block = saved_bl;
        return rc ? rc : DIRAC_ERR_INVALID_ARG;
    }
    op->vr = best->vr;
    op->minb = best->minb;
    op->block = best->block;
    remember_tuning(op);
    if (best_ms) *best_ms = best->ms;
    return DIRAC_OK;
}

static int apply_checked(const dirac_op *op, const void *in, void *out, double m0, int sgn, void *stream) {
    if (!op) return DIRAC_ERR_INVALID_ARG;
    int rc = check_vec(in);
    if (!rc) rc = check_vec(out);
    if (rc) return rc;
    if (in == out) return DIRAC_ERR_INVALID_ARG;
    return op_apply(op, in, out, m0, sgn, (cudaStream_t)stream);
}

int dirac_apply(const dirac_op *op, const void *psi_in, void *psi_out, double m0, void *stream) {
    return apply_checked(op, psi_in, psi_out, m0, +1, stream);
}

int dirac_apply_dagger(const dirac_op *op, const void *psi_in, void *psi_out, double m0, void *stream) {
    return apply_checked(op, psi_in, psi_out, m0, -1, stream);
}

int dirac_apply_normal(const dirac_op *op, const void *psi_in, void *psi_out, double m0, void *stream) {
    if (!op) return DIRAC_ERR_INVALID_ARG;
    int rc = check_vec(psi_in);
    if (!rc) rc = check_vec(psi_out);
    if (rc) return rc;
    return op_apply_normal(op, psi_in, psi_out, m0, (cudaStream_t)stream);
}

// Copy the sites of time slices [t0, t1) of a vector between host and device
// (same offsets on both sides): one run for the site-outer layout, one run per
// internal component for the site-inner layout.
static int copy_slab(const dirac_op *op, void *dst, const void *src, int t0, int t1, cudaMemcpyKind kind,
                     cudaStream_t s) {
    const size_t per_site = (size_t)op->nv * 2 * elem_bytes(op->prec);
    const size_t ncs = (size_t)(op->rows / op->V);
    const size_t slab_sites = (size_t)op->lat.nx * op->lat.ny * op->lat.nz;
    const size_t first = (size_t)t0 * slab_sites, count = (size_t)(t1 - t0) * slab_sites;
    if (op->geom.layout == DIRAC_LAYOUT_SITE_OUTER) {
        const size_t off = first * ncs * per_site;
        return cuda_check(cudaMemcpyAsync((char *)dst + off, (const char *)src + off, count * ncs * per_site, kind, s),
                          "slab copy");
    }
    const size_t pitch = (size_t)op->V * per_site, off = first * per_site;
    if (pitch < ((size_t)1 << 31))
        return cuda_check(cudaMemcpy2DAsync((char *)dst + off, pitch, (const char *)src + off, pitch, count * per_site,
                                            ncs, kind, s),
                          "slab copy");
    for (size_t c = 0; c < ncs; ++c) {
        const size_t o = c * pitch + off;
        const int rc = cuda_check(cudaMemcpyAsync((char *)dst + o, (const char *)src + o, count * per_site, kind, s),
                                  "slab copy");
        if (rc) return rc;
    }
    return DIRAC_OK;
}

static int host_apply(const dirac_op *op, const void *host_in, void *host_out, double m0, int dagger, void *stream,
                      bool sync) {
    if (!op || !host_in || !host_out) return DIRAC_ERR_INVALID_ARG;
    dirac_op *self = (dirac_op *)op;
    int rc = DIRAC_OK;
    if (!self->stage_in) rc = alloc(&self->stage_in, op->vec_bytes);
    if (!rc && !self->stage_out) rc = alloc(&self->stage_out, op->vec_bytes);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const int sgn = dagger ? -1 : +1;
    const int nt = op->lat.nt;
    const int K = nt < kMaxSlabs ? nt : kMaxSlabs;   // slabs of whole time slices
    if (K < 3) {
        rc = cuda_check(cudaMemcpyAsync(self->stage_in, host_in, op->vec_bytes, cudaMemcpyHostToDevice, s), "H2D");
        if (!rc) rc = op_apply(op, self->stage_in, self->stage_out, m0, sgn, s);
        if (!rc) rc = cuda_check(cudaMemcpyAsync(host_out, self->stage_out, op->vec_bytes, cudaMemcpyDeviceToHost, s),
                                 "D2H");
        if (!rc && sync) rc = cuda_check(cudaStreamSynchronize(s), "apply_host sync");
        return rc;
    }
    // Pipelined: slab k = time slices [k nt / K, (k+1) nt / K) goes in on the
    // copy-in stream; the output of slab k needs the input of slabs k-1, k,
    // k+1 (every stencil reaches one slice in t), so the stencil runs on slabs
    // 1, 2, .., K-1 as their upper neighbours arrive and on slab 0 last; each
    // finished output slab goes out on the copy-out stream while later slabs
    // are still being copied in or computed.  The synchronous form runs the
    // stencils on `stream`; the asynchronous one on the operator's own compute
    // stream, so that its stencils do not queue behind the copies out of
    // another operator's host apply that `stream` waits for.
    dirac_host_pipe *p = nullptr;
    CTRY(pipe_get(self, &p));
    cudaStream_t cs = sync ? s : p->comp;
    auto t_of = [&](int k) { return (int)((long long)k * nt / K); };
    if (sync) {
        CTRY(cuda_check(cudaEventRecord(p->start, s), "pipe event"));      // staging buffers free
        CTRY(cuda_check(cudaStreamWaitEvent(p->h2d, p->start, 0), "pipe wait"));
        CTRY(cuda_check(cudaStreamWaitEvent(p->d2h, p->start, 0), "pipe wait"));
    } else if (p->used) {
        // asynchronous form: the staging buffers are free once this
        // operator's previous host apply has copied its output out; earlier
        // work of other operators on `stream` is not waited for, so their
        // computation overlaps these copies
        CTRY(cuda_check(cudaStreamWaitEvent(p->h2d, p->end, 0), "pipe wait"));
    }
    for (int k = 0; k < K; ++k) {
        CTRY(copy_slab(op, self->stage_in, host_in, t_of(k), t_of(k + 1), cudaMemcpyHostToDevice, p->h2d));
        CTRY(cuda_check(cudaEventRecord(p->in_done[k], p->h2d), "pipe event"));
    }
    const long long slab_sites = (long long)op->lat.nx * op->lat.ny * op->lat.nz;
    for (int i = 0; i < K; ++i) {
        const int k = (i + 1) % K;
        const int need = (k >= 1 && k <= K - 2) ? k + 1 : K - 1;   // last input slab it reads
        CTRY(cuda_check(cudaStreamWaitEvent(cs, p->in_done[need], 0), "pipe wait"));
        dirac_op part = *op;   // same buffers, output sites of slab k only
        part.lat.n0 = t_of(k) * slab_sites;
        part.lat.nsites = (t_of(k + 1) - t_of(k)) * slab_sites;
        CTRY(op_apply(&part, self->stage_in, self->stage_out, m0, sgn, cs));
        CTRY(cuda_check(cudaEventRecord(p->out_ready[k], cs), "pipe event"));
        CTRY(cuda_check(cudaStreamWaitEvent(p->d2h, p->out_ready[k], 0), "pipe wait"));
        CTRY(copy_slab(op, host_out, self->stage_out, t_of(k), t_of(k + 1), cudaMemcpyDeviceToHost, p->d2h));
    }
    CTRY(cuda_check(cudaEventRecord(p->end, p->d2h), "pipe event"));
    p->used = true;
    CTRY(cuda_check(cudaStreamWaitEvent(s, p->end, 0), "pipe wait"));
    return sync ? cuda_check(cudaStreamSynchronize(s), "apply_host sync") : DIRAC_OK;
}

int dirac_apply_host(const dirac_op *op, const void *host_in, void *host_out, double m0, int dagger, void *stream) {
    return host_apply(op, host_in, host_out, m0, dagger, stream, true);
}

int dirac_apply_host_async(const dirac_op *op, const void *host_in, void *host_out, double m0, int dagger,
                           void *stream) {
    return host_apply(op, host_in, host_out, m0, dagger, stream, false);
}

int dirac_vec_norm2(const dirac_op *op, const void *v, double *out_dev, void *stream) {
    if (!op || !out_dev) return DIRAC_ERR_INVALID_ARG;
    int rc = check_vec(v);
    return rc ? rc : blas_norm2(op, op->prec, v, out_dev, (cudaStream_t)stream);
}

int dirac_vec_dot(const dirac_op *op, const void *u, const void *v, double *out_dev, void *stream) {
    if (!op || !out_dev) return DIRAC_ERR_INVALID_ARG;
    int rc = check_vec(u);
    if (!rc) rc = check_vec(v);
    return rc ? rc : blas_dot(op, op->prec, u, v, out_dev, (cudaStream_t)stream);
}

int dirac_vec_axpy(const dirac_op *op, const double *alpha_dev, const void *x, void *y, void *stream) {
    if (!op || !alpha_dev) return DIRAC_ERR_INVALID_ARG;
    int rc = check_vec(x);
    if (!rc) rc = check_vec(y);
    return rc ? rc : blas_axpy(op, op->prec, alpha_dev, x, y, (cudaStream_t)stream);
}

int dirac_vec_axpby(const dirac_op *op, const double *a_dev, const void *x, const double *b_dev, const void *y,
                    void *z, void *stream) {
    if (!op || !a_dev || !b_dev) return DIRAC_ERR_INVALID_ARG;
    int rc = check_vec(x);
    if (!rc) rc = check_vec(y);
    if (!rc) rc = check_vec(z);
    return rc ? rc : blas_axpby(op, op->prec, z, x, a_dev, 1.0, y, b_dev, 1.0, nullptr, (cudaStream_t)stream);
}

static int check_range(const dirac_op *op, long long site0, long long nsites) {
    return (site0 < 0 || nsites < 1 || site0 + nsites > op->V) ? DIRAC_ERR_INVALID_ARG : DIRAC_OK;
}

int dirac_vec_norm2_range(const dirac_op *op, const void *v, long long site0, long long nsites, double *out_dev,
                          void *stream) {
    if (!op || !out_dev) return DIRAC_ERR_INVALID_ARG;
    int rc = check_vec(v);
    if (!rc) rc = check_range(op, site0, nsites);
    return rc ? rc : blas_norm2_range(op, op->prec, v, site0, nsites, out_dev, (cudaStream_t)stream);
}

int dirac_vec_dot_range(const dirac_op *op, const void *u, const void *v, long long site0, long long nsites,
                        double *out_dev, void *stream) {
    if (!op || !out_dev) return DIRAC_ERR_INVALID_ARG;
    int rc = check_vec(u);
    if (!rc) rc = check_vec(v);
    if (!rc) rc = check_range(op, site0, nsites);
    return rc ? rc : blas_dot_range(op, op->prec, u, v, site0, nsites, out_dev, (cudaStream_t)stream);
}

int dirac_vec_gamma5(const dirac_op *op, void *v, void *stream) {
    if (!op) return DIRAC_ERR_INVALID_ARG;
    int rc = check_vec(v);
    return rc ? rc : blas_gamma5(op, op->prec, v, (cudaStream_t)stream);
}

int dirac_vec_convert(const dirac_op *op, const void *src, dirac_prec src_prec, void *dst, dirac_prec dst_prec,
                      void *stream) {
    if (!op) return DIRAC_ERR_INVALID_ARG;
    if (src_prec < DIRAC_F64 || src_prec > DIRAC_F16 || dst_prec < DIRAC_F64 || dst_prec > DIRAC_F16)
        return DIRAC_ERR_UNSUPPORTED_PREC;
    int rc = check_vec(src);
    if (!rc) rc = check_vec(dst);
    return rc ? rc : blas_convert(op, src, src_prec, dst, dst_prec, (cudaStream_t)stream);
}

const char *dirac_error_string(int code) {
    switch (code) {
    case DIRAC_OK: return "success";
    case DIRAC_ERR_INVALID_ARG: return "invalid argument";
    case DIRAC_ERR_UNSUPPORTED_NC: return "unsupported number of colours";
    case DIRAC_ERR_UNSUPPORTED_PREC: return "unsupported precision";
    case DIRAC_ERR_ALIGNMENT: return "vector pointer not 16-byte aligned";
    case DIRAC_ERR_OOM: return "device allocation failed";
    case DIRAC_ERR_CUDA: return "CUDA error";
    case DIRAC_ERR_DEVICE_TIMEOUT: return "bounded device wait timed out";
    case DIRAC_ERR_CAPACITY: return "request exceeds a fixed static capacity";
    case DIRAC_NOT_CONVERGED: return "solver reached maxit";
    case DIRAC_STAGNATED: return "solver stagnated (updated vs recomputed residual differ by >1%)";
    case DIRAC_BREAKDOWN: return "solver breakdown";
    case DIRAC_NONFINITE: return "non-finite residual";
    }
    return "unknown code";
}

long dirac_clover_flops_per_site(int nc) { return 64L * nc * nc; }

long dirac_flops_per_site(dirac_kind kind, int nc) {
    const long n = nc;
    switch (kind) {
    case DIRAC_WILSON: return 128 * n * n + 72 * n;
    case DIRAC_BRILLOUIN: return 2560 * n * n + 2376 * n;
    case DIRAC_STAGGERED: return 64 * n * n + 2 * n;
    case DIRAC_WLAP: return 256 * n * n + 8 * n;
    case DIRAC_BLAP: return 2560 * n * n + 648 * n;
    case DIRAC_WSUV: return 64 * n * n + 2 * n;
    case DIRAC_BSUV: return 640 * n * n + 162 * n;
    }
    return -1;
}

int dirac_version(void) { return 100; }

}  // extern "C"
