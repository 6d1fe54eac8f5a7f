// batch.cu -- many independent multi-RHS CG solves in one CUDA graph.
//
// Each solve (its own operator handle: lattice, N_v, links, workspace) runs
// CG on D^dag D with every coefficient, mask and convergence decision kept on
// the device, so an iteration is a host-free chain of kernels.  A segment of
// K iterations followed by the recompute of the true residual (the paper's
// recompute rule, Sec. 9, every K = 20 iterations in low precision) is
// recorded per solve into the body of a conditional (if) node; the if nodes
// of all solves sit side by side (small lattices run concurrently) in the
// body of one while node, closed by a kernel that keeps the loop going while
// any solve is unconverged.  The host launches that graph once and waits
// once; the loop, the per-solve skipping of converged solves and the
// convergence test all run on the device.  A solve's completion is stamped
// on the device with %globaltimer.  No kernel waits on another: ordering
// comes only from graph edges and the conditional nodes.  Where the driver
// cannot build conditional nodes, a host loop replays a one-segment graph
// instead (stats report the number of host launches).
#include <math.h>
#include <string.h>

#include <chrono>
#include <vector>

#include "internal.h"

namespace dgb {

int solver_ws(const dirac_op *op, void **vecs, int nvecs, double **scal);
int batch_apply_A_pq(const dirac_op *op, const void *p, void *q, double *pq, double m0, cudaStream_t s);

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void stamp_kernel(unsigned long long *t) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *t = globaltimer();
}

// pq holds N_v real values |D p|^2
__global__ void batch_alpha_kernel(int nv, const double *rr, const double *pq, const double *act, double *alpha) {
    const int v = threadIdx.x;
    if (v >= nv) return;
    const double p = pq[v];
    const double a = (act[v] != 0.0 && p > 0.0) ? rr[v] / p : 0.0;
    alpha[2 * v] = a;
    alpha[2 * v + 1] = 0.0;
}

__global__ void batch_beta_kernel(int nv, const double *rr_new, double *rr, const double *act, double *beta) {
    const int v = threadIdx.x;
    if (v >= nv) return;
    const double b = (act[v] != 0.0 && rr[v] > 0.0) ? rr_new[v] / rr[v] : 0.0;
    beta[2 * v] = b;
    beta[2 * v + 1] = 0.0;
    rr[v] = rr_new[v];
}

// After a recompute: freeze the RHS whose true residual passes; when all have
// passed, mark the solve done and stamp the time (first time only).
struct BatchState {
    int done;
    int iters;
    unsigned long long stamp;
};

__global__ void batch_check_kernel(int nv, const double *rr_true, const double *nb, double tol2, double *act,
                                   BatchState *st, int K, cudaGraphConditionalHandle cond, int set_cond) {
    __shared__ int any;
    const int v = threadIdx.x;
    if (v == 0) any = 0;
    __syncthreads();
    const int done = st->done;
    if (v < nv && !done) {
        const bool pass = !(rr_true[v] >= tol2 * nb[v]);
        act[v] = pass ? 0.0 : 1.0;
        if (!pass) atomicOr(&any, 1);
    }
    __syncthreads();
    if (v == 0 && !done) {
        st->iters += K;
        if (!any) {
            st->done = 1;
            st->stamp = globaltimer();
        }
    }
    // inside the device-side loop: this solve's segment runs again only while
    // it has not converged
    if (v == 0 && set_cond) cudaGraphSetConditional(cond, st->done ? 0u : 1u);
}

// End of one pass of the device-side loop: another pass while any solve is
// unconverged and the iteration limit allows (a single thread; one launch).
__global__ void batch_while_kernel(const BatchState *st, int nsolves, int *passes, int max_passes,
                                   cudaGraphConditionalHandle cond) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int any = 0;
    for (int i = 0; i < nsolves; ++i) any |= st[i].done == 0;
    const int p = ++*passes;
    cudaGraphSetConditional(cond, (any && p < max_passes) ? 1u : 0u);
}

}  // namespace dgb

using namespace dgb;

#define TRYB(x)                 \
    do {                        \
        int rc_ = (x);          \
        if (rc_) {              \
            rc = rc_;           \
            goto fail;          \
        }                       \
    } while (0)

extern "C" int dirac_solve_batched(int nsolves, dirac_op *const *ops, const void *const *b, void *const *x,
                                   const double *m0, const dirac_solve_params *prm, dirac_solve_stats *stats,
                                   void *stream) {
    if (nsolves < 1 || nsolves > 1024 || !ops || !b || !x || !m0 || !prm) return DIRAC_ERR_INVALID_ARG;
    if (prm->solver != DIRAC_CG_NORMAL && prm->solver != DIRAC_CG_HPD) return DIRAC_ERR_INVALID_ARG;
    if (!(prm->tol > 0) || prm->maxit < 1) return DIRAC_ERR_INVALID_ARG;
    for (int i = 0; i < nsolves; ++i) {
        if (!ops[i] || !b[i] || !x[i]) return DIRAC_ERR_INVALID_ARG;
        if (((uintptr_t)b[i] & 15) || ((uintptr_t)x[i] & 15)) return DIRAC_ERR_ALIGNMENT;
        if (prm->inner_prec != ops[i]->prec) return DIRAC_ERR_UNSUPPORTED_PREC;   // one precision per solve
        if (is_laplace(ops[i]->kind) && prm->solver == DIRAC_CG_NORMAL) return DIRAC_ERR_INVALID_ARG;
        for (int j = 0; j < i; ++j)
            if (ops[j] == ops[i]) return DIRAC_ERR_INVALID_ARG;   // each solve owns its workspace
    }
    // all work runs on a private non-blocking stream ordered after the
    // caller's stream (the legacy default stream cannot be captured)
    cudaStream_t user = (cudaStream_t)stream;
    cudaStream_t main = nullptr;
    cudaEvent_t entry = nullptr;
    const int K = prm->recompute_every > 0 ? prm->recompute_every : 20;
    const double tol2 = prm->tol * prm->tol;
    std::vector<cudaStream_t> br(nsolves, nullptr);
    std::vector<cudaEvent_t> joins(nsolves, nullptr);
    cudaEvent_t fork = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    BatchState *dstate = nullptr;
    unsigned long long *dstart = nullptr;
    std::vector<BatchState> hstate(nsolves);
    unsigned long long hstart = 0;
    std::vector<void *> vecs(nsolves * 4);
    std::vector<double *> scal(nsolves);
    int rc = DIRAC_OK, replays = 0;
    const int max_replays = (prm->maxit + K - 1) / K;
    auto t0 = std::chrono::steady_clock::now();

    // per solve: rhs (vec 3), r (0), p (1), q (2); scalars: rr, rr_new, pq, alpha, beta, act, nb
    TRYB(cuda_check(cudaStreamCreateWithFlags(&main, cudaStreamNonBlocking), "stream"));
    TRYB(cuda_check(cudaEventCreateWithFlags(&entry, cudaEventDisableTiming), "event"));
    TRYB(cuda_check(cudaEventRecord(entry, user), "entry"));
    TRYB(cuda_check(cudaStreamWaitEvent(main, entry, 0), "wait entry"));
    for (int i = 0; i < nsolves; ++i) {
        void *v4[4];
        double *sc = nullptr;
        TRYB(solver_ws(ops[i], v4, 4, &sc));
        for (int k = 0; k < 4; ++k) vecs[i * 4 + k] = v4[k];
        scal[i] = sc;
    }
    TRYB(cuda_check(cudaMalloc(&dstate, nsolves * sizeof(BatchState)), "batch state"));
    TRYB(cuda_check(cudaMalloc(&dstart, sizeof(unsigned long long)), "batch stamp"));
    TRYB(cuda_check(cudaMemsetAsync(dstate, 0, nsolves * sizeof(BatchState), main), "memset"));
    TRYB(cuda_check(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming), "event"));
    for (int i = 0; i < nsolves; ++i) {
        TRYB(cuda_check(cudaStreamCreateWithFlags(&br[i], cudaStreamNonBlocking), "stream"));
        TRYB(cuda_check(cudaEventCreateWithFlags(&joins[i], cudaEventDisableTiming), "event"));
    }
    stamp_kernel<<<1, 1, 0, main>>>(dstart);
    // set-up on the main stream: rhs, r = rhs - A x, p = r, norms, masks
    for (int i = 0; i < nsolves; ++i) {
        const dirac_op *op = ops[i];
        const dirac_prec p = op->prec;
        const int nv = op->nv;
        void *r = vecs[i * 4 + 0], *pv = vecs[i * 4 + 1], *q = vecs[i * 4 + 2], *rhs = vecs[i * 4 + 3];
        double *sc = scal[i];
        double *rr = sc, *nb = sc + 6 * 128, *act = sc + 5 * 128;
        if (prm->solver == DIRAC_CG_NORMAL) TRYB(op_apply(op, b[i], rhs, m0[i], -1, main));
        else TRYB(blas_axpby(op, p, rhs, b[i], nullptr, 1.0, nullptr, nullptr, 0.0, nullptr, main));
        TRYB(blas_norm2(op, p, rhs, nb, main));
        TRYB(op_apply_cg(op, x[i], q, m0[i], main));
        TRYB(blas_axpby(op, p, r, rhs, nullptr, 1.0, q, nullptr, -1.0, rr, main));
        TRYB(blas_axpby(op, p, pv, r, nullptr, 1.0, nullptr, nullptr, 0.0, nullptr, main));
        batch_check_kernel<<<1, 64, 0, main>>>(nv, rr, nb, tol2, act, dstate + i, 0, 0, 0);
        TRYB(launch_check("batch setup"));
    }
    TRYB(cuda_check(cudaMemcpyAsync(hstate.data(), dstate, nsolves * sizeof(BatchState), cudaMemcpyDeviceToHost,
                                    main), "D2H state"));
    TRYB(cuda_check(cudaStreamSynchronize(main), "batch sync"));
    {
        // one segment (K iterations + recompute + convergence check) of solve i on stream s
        auto record_segment = [&](int i, cudaStream_t s, cudaGraphConditionalHandle cond, int set_cond) -> int {
            const dirac_op *op = ops[i];
            const dirac_prec p = op->prec;
            const int nv = op->nv;
            void *r = vecs[i * 4 + 0], *pv = vecs[i * 4 + 1], *q = vecs[i * 4 + 2], *rhs = vecs[i * 4 + 3];
            double *sc = scal[i];
            double *rr = sc, *rr_new = sc + 128, *pq = sc + 2 * 128, *alpha = sc + 3 * 128, *beta = sc + 4 * 128;
            double *act = sc + 5 * 128, *nb = sc + 6 * 128;
            int e;
            for (int k = 0; k < K; ++k) {
                if ((e = batch_apply_A_pq(op, pv, q, pq, m0[i], s))) return e;
                batch_alpha_kernel<<<1, 64, 0, s>>>(nv, rr, pq, act, alpha);
                if ((e = blas_axpby(op, p, r, r, nullptr, 1.0, q, alpha, -1.0, rr_new, s))) return e;
                if (k + 1 < K) {
                    batch_beta_kernel<<<1, 64, 0, s>>>(nv, rr_new, rr, act, beta);
                    if ((e = blas_update_xp(op, p, x[i], pv, r, alpha, beta, s))) return e;   // x += alpha p; p = r + beta p
                } else {
                    // last iteration of the segment: x += alpha p, then replace r by
                    // the true residual and build the next direction from it
                    if ((e = blas_axpby(op, p, x[i], x[i], nullptr, 1.0, pv, alpha, 1.0, nullptr, s))) return e;
                    if ((e = op_apply_cg(op, x[i], q, m0[i], s))) return e;
                    if ((e = blas_axpby(op, p, r, rhs, nullptr, 1.0, q, nullptr, -1.0, rr_new, s))) return e;
                    batch_beta_kernel<<<1, 64, 0, s>>>(nv, rr_new, rr, act, beta);
                    if ((e = blas_axpby(op, p, pv, r, nullptr, 1.0, pv, beta, 1.0, nullptr, s))) return e;
                }
            }
            // freeze converged RHS (rr now holds the true residual), stamp completion
            batch_check_kernel<<<1, 64, 0, s>>>(nv, rr, nb, tol2, act, dstate + i, K, cond, set_cond);
            return launch_check("batch segment");
        };

        // Device-side loop: one graph whose while node repeats, until every
        // solve has converged or the iteration limit is reached, a body that
        // holds one conditional (if) node per solve, each running that
        // solve's segment only while it is unconverged.  The host launches it
        // once and waits once.  If the driver cannot build it, the host
        // replay below runs the same segments instead.
        bool device_loop = false;
        {
            cudaGraph_t g = nullptr;
            cudaGraphExec_t gx = nullptr;
            int *dpasses = nullptr;
            int e = cuda_check(cudaMalloc(&dpasses, sizeof(int)), "pass counter");
            if (!e) e = cuda_check(cudaMemsetAsync(dpasses, 0, sizeof(int), main), "memset");
            if (!e) e = cuda_check(cudaGraphCreate(&g, 0), "graph create");
            cudaGraphConditionalHandle hw = 0;
            cudaGraph_t body = nullptr;
            if (!e) e = cuda_check(cudaGraphConditionalHandleCreate(&hw, g, 1, cudaGraphCondAssignDefault),
                                   "while handle");
            if (!e) {
                cudaGraphNodeParams wp = {};
                wp.type = cudaGraphNodeTypeConditional;
                wp.conditional.handle = hw;
                wp.conditional.type = cudaGraphCondTypeWhile;
                wp.conditional.size = 1;
                cudaGraphNode_t wnode;
                e = cuda_check(cudaGraphAddNode(&wnode, g, nullptr, nullptr, 0, &wp), "while node");
                if (!e) body = wp.conditional.phGraph_out[0];
            }
            std::vector<cudaGraphNode_t> ifs(nsolves);
            for (int i = 0; i < nsolves && !e; ++i) {
                cudaGraphConditionalHandle hi = 0;
                e = cuda_check(cudaGraphConditionalHandleCreate(&hi, body, hstate[i].done ? 0 : 1,
                                                                cudaGraphCondAssignDefault), "if handle");
                if (e) break;
                cudaGraphNodeParams ip = {};
                ip.type = cudaGraphNodeTypeConditional;
                ip.conditional.handle = hi;
                ip.conditional.type = cudaGraphCondTypeIf;
                ip.conditional.size = 1;
                e = cuda_check(cudaGraphAddNode(&ifs[i], body, nullptr, nullptr, 0, &ip), "if node");
                if (e) break;
                e = cuda_check(cudaStreamBeginCaptureToGraph(br[i], ip.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                             cudaStreamCaptureModeThreadLocal), "capture to graph");
                if (e) break;
                const int seg = record_segment(i, br[i], hi, 1);
                cudaGraph_t captured = nullptr;
                const int end_rc = cuda_check(cudaStreamEndCapture(br[i], &captured), "end capture");
                e = seg ? seg : end_rc;
            }
            if (!e) {
                cudaKernelNodeParams kp = {};
                int ns = nsolves, maxp = max_replays;
                void *args[] = {(void *)&dstate, (void *)&ns, (void *)&dpasses, (void *)&maxp, (void *)&hw};
                kp.func = (void *)batch_while_kernel;
                kp.gridDim = dim3(1);
                kp.blockDim = dim3(32);
                kp.kernelParams = args;
                cudaGraphNode_t kn;
                e = cuda_check(cudaGraphAddKernelNode(&kn, body, ifs.data(), nsolves, &kp), "while kernel node");
            }
            if (!e) e = cuda_check(cudaGraphInstantiate(&gx, g, 0), "graph instantiate");
            if (!e) {
                device_loop = true;
                rc = cuda_check(cudaGraphLaunch(gx, main), "graph launch");
                ++replays;
                if (!rc) rc = cuda_check(cudaMemcpyAsync(hstate.data(), dstate, nsolves * sizeof(BatchState),
                                                         cudaMemcpyDeviceToHost, main), "D2H state");
                if (!rc) rc = cuda_check(cudaStreamSynchronize(main), "batch sync");
            }
            if (gx) cudaGraphExecDestroy(gx);
            if (g) cudaGraphDestroy(g);
            if (dpasses) {
                cudaStreamSynchronize(main);
                cudaFree(dpasses);
            }
            cudaGetLastError();
            if (device_loop && rc) goto fail;
            rc = DIRAC_OK;
        }

        // Host replay: the graph holds one segment of every solve still
        // running; it is rebuilt without the finished ones whenever a solve
        // completes, so converged solves stop costing GPU time.
        while (!device_loop && replays < max_replays) {
            std::vector<int> live;
            for (int i = 0; i < nsolves; ++i)
                if (!hstate[i].done) live.push_back(i);
            if (live.empty()) break;
            TRYB(cuda_check(cudaStreamBeginCapture(main, cudaStreamCaptureModeThreadLocal), "begin capture"));
            TRYB(cuda_check(cudaEventRecord(fork, main), "fork"));
            for (int i : live) {
                TRYB(cuda_check(cudaStreamWaitEvent(br[i], fork, 0), "wait fork"));
                TRYB(record_segment(i, br[i], 0, 0));
                TRYB(cuda_check(cudaEventRecord(joins[i], br[i]), "join"));
                TRYB(cuda_check(cudaStreamWaitEvent(main, joins[i], 0), "wait join"));
            }
            rc = cuda_check(cudaStreamEndCapture(main, &graph), "end capture");
            if (rc) goto fail;
            TRYB(cuda_check(cudaGraphInstantiate(&exec, graph, 0), "graph instantiate"));
            for (; replays < max_replays; ++replays) {
                TRYB(cuda_check(cudaGraphLaunch(exec, main), "graph launch"));
                TRYB(cuda_check(cudaMemcpyAsync(hstate.data(), dstate, nsolves * sizeof(BatchState),
                                                cudaMemcpyDeviceToHost, main), "D2H state"));
                TRYB(cuda_check(cudaStreamSynchronize(main), "batch sync"));
                bool finished_one = false;
                for (int i : live) finished_one |= hstate[i].done != 0;
                if (finished_one) {
                    ++replays;
                    break;
                }
            }
            cudaGraphExecDestroy(exec);
            exec = nullptr;
            cudaGraphDestroy(graph);
            graph = nullptr;
        }
    }
    TRYB(cuda_check(cudaMemcpy(&hstart, dstart, sizeof(hstart), cudaMemcpyDeviceToHost), "D2H stamp"));
    if (stats) {
        const double wall = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        for (int i = 0; i < nsolves; ++i) {
            dirac_solve_stats &st = stats[i];
            memset(&st, 0, sizeof(st));
            const int nv = ops[i]->nv;
            double rr[64], nb[64];
            TRYB(cuda_check(cudaMemcpy(rr, scal[i], nv * sizeof(double), cudaMemcpyDeviceToHost), "D2H"));
            TRYB(cuda_check(cudaMemcpy(nb, scal[i] + 6 * 128, nv * sizeof(double), cudaMemcpyDeviceToHost), "D2H"));
            st.iters = hstate[i].iters;
            st.recomputes = hstate[i].iters / K;
            st.status = hstate[i].done ? DIRAC_OK : DIRAC_NOT_CONVERGED;
            for (int v = 0; v < nv; ++v) {
                st.relres[v] = nb[v] > 0 ? sqrt(rr[v] / nb[v]) : 0.0;
                st.status_per_rhs[v] = (nb[v] == 0.0 || rr[v] < tol2 * nb[v]) ? DIRAC_OK : DIRAC_NOT_CONVERGED;
            }
            st.seconds = hstate[i].done ? (double)(hstate[i].stamp - hstart) * 1e-9 : wall;
            st.host_launches = replays;
        }
    }
    rc = DIRAC_OK;
    {
        bool all = true;
        for (int i = 0; i < nsolves; ++i) all &= hstate[i].done != 0;
        if (!all) rc = DIRAC_NOT_CONVERGED;
    }
fail:
    if (main) {
        cudaStreamCaptureStatus cs;
        if (cudaStreamIsCapturing(main, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
            cudaGraph_t g2 = nullptr;
            cudaStreamEndCapture(main, &g2);
            if (g2) cudaGraphDestroy(g2);
            if (!rc) rc = DIRAC_ERR_CUDA;
        }
    }
    cudaGetLastError();
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (int i = 0; i < nsolves; ++i) {
        if (joins[i]) cudaEventDestroy(joins[i]);
        if (br[i]) cudaStreamDestroy(br[i]);
    }
    if (fork) cudaEventDestroy(fork);
    if (main) {
        cudaStreamSynchronize(main);
        cudaStreamDestroy(main);
    }
    if (entry) cudaEventDestroy(entry);
    cudaFree(dstate);
    cudaFree(dstart);
    return rc;
}
