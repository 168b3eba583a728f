// Solvers (Section 6): even-odd preconditioned BiCGstab with FP64 defect
// correction around a reduced-precision inner loop, the multi-mass driver
// with the Lagrange initial guess, and the plumbing they share.
//
// Inner BiCGstab iteration on M_prec = 1 - kappa^2 D_eo D_oe, per rhs
// (van der Vorst; the paper cites it and does not print it):
//   v = M_prec p                 hop D_oe p -> tmp;  v = p - k^2 D_eo tmp, <rhat,v> -> alpha
//   s = r - alpha v
//   t = M_prec s                 hop D_oe s -> tmp;  t = s - k^2 D_eo tmp, <t,s>, <t,t> -> omega
//   x += alpha p + omega s; r = s - omega t;   <rhat,r>, ||r||^2 -> beta, convergence
//   p = r + beta (p - omega v)
// Seven kernels; every scalar stays in device memory (BiState), so an
// iteration needs no host round trip and a block of iterations can be
// replayed from a captured CUDA graph.  Kernels of a converged rhs return
// at once, so surplus captured iterations cost only empty launches.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "internal.h"

namespace wl {

// Scratch of one batched solve: per-rhs state, reduction partials, flags.
struct Scratch {
    BiState *state = nullptr;    // [nrhs]
    double *partials = nullptr;  // [nrhs][2 * site_blocks][kRedNV]
    double *norms = nullptr;     // [nrhs * 4]
    unsigned *tickets = nullptr; // [nrhs * 4]
    int *active = nullptr;       // [nrhs]
    double *delta2 = nullptr;    // [nrhs]
    double *coef = nullptr;      // [4][nrhs * 32] lincomb coefficients (two sets, re and im)
    double *kappa2 = nullptr;    // [1] -kappa^2 of the current mass (read by graph-captured kernels)
    int *outer_done = nullptr;   // [nrhs] 1 once the outer residual of rhs r has converged
};

static int get_scratch(wl_gauge *g, int nrhs, Scratch *sc, cudaStream_t s)
{
    const Geom &geo = g->lat->geom;
    void *p;
    WL_TRY(g->ws.get("state", sizeof(BiState) * nrhs, &p));
    sc->state = static_cast<BiState *>(p);
    WL_TRY(g->ws.get("partials", sizeof(double) * nrhs * 2 * site_blocks(geo) * kRedNV, &p));
    sc->partials = static_cast<double *>(p);
    WL_TRY(g->ws.get("norms", sizeof(double) * nrhs * 4, &p));
    sc->norms = static_cast<double *>(p);
    bool fresh = g->ws.bufs["tickets"].bytes < sizeof(unsigned) * nrhs * 4;
    WL_TRY(g->ws.get("tickets", sizeof(unsigned) * nrhs * 4, &p));
    sc->tickets = static_cast<unsigned *>(p);
    if (fresh) WL_CUDA_TRY(cudaMemsetAsync(p, 0, sizeof(unsigned) * nrhs * 4, s));
    WL_TRY(g->ws.get("active", sizeof(int) * nrhs, &p));
    sc->active = static_cast<int *>(p);
    WL_TRY(g->ws.get("delta2", sizeof(double) * nrhs, &p));
    sc->delta2 = static_cast<double *>(p);
    WL_TRY(g->ws.get("coef", sizeof(double) * 4 * nrhs * 32, &p));
    sc->coef = static_cast<double *>(p);
    WL_TRY(g->ws.get("kappa2", sizeof(double), &p));
    sc->kappa2 = static_cast<double *>(p);
    WL_TRY(g->ws.get("outer_done", sizeof(int) * nrhs, &p));
    sc->outer_done = static_cast<int *>(p);
    // tickets inside BiState start at zero
    WL_CUDA_TRY(cudaMemsetAsync(sc->state, 0, sizeof(BiState) * nrhs, s));
    return WL_OK;
}

void GraphCache::release()
{
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    for (auto e : events) cudaEventDestroy(e);
    events.clear();
    key.clear();
    kernels = 0;
}

// --------------------------------------------------------------- inner loop

struct Inner {
    wl_gauge *g;
    int prec, xprec, nrhs;
    double kappa;
    Vec r, rhat, p, v, s, t, tmp, e;
    Scratch sc;
};

static int make_inner(wl_gauge *g, int prec, int nrhs, double kappa, Inner *in, cudaStream_t s)
{
    in->g = g;
    in->prec = prec;
    in->xprec = prec == WL_F64 ? WL_F64 : WL_F32;
    in->nrhs = nrhs;
    in->kappa = kappa;
    WL_TRY(make_vec(g, "in_r", prec, nrhs, &in->r));
    WL_TRY(make_vec(g, "in_rhat", prec, nrhs, &in->rhat));
    WL_TRY(make_vec(g, "in_p", prec, nrhs, &in->p));
    WL_TRY(make_vec(g, "in_v", prec, nrhs, &in->v));
    WL_TRY(make_vec(g, "in_s", prec, nrhs, &in->s));
    WL_TRY(make_vec(g, "in_t", prec, nrhs, &in->t));
    WL_TRY(make_vec(g, "in_tmp", prec, nrhs, &in->tmp));
    WL_TRY(make_vec(g, "in_e", in->xprec, nrhs, &in->e));
    return get_scratch(g, nrhs, &in->sc, s);
}

// z = M^dag r with ||z||^2 and beta, then p = z + beta p (CG on the normal
// equations; after a restart beta = 0, so p = z).
static int cg_normal_residual(Inner &in, int rhs_block, cudaStream_t s)
{
    const Geom &geo = in.g->lat->geom;
    const int *skip = &in.sc.state[0].done;
    const int ss = sizeof(BiState) / sizeof(int);
    WL_TRY(hop_ex(in.g, in.r, in.tmp, nullptr, 0.0, nullptr, 0.0, 1.0, WL_ODD, 1, rhs_block, skip, ss, s));
    WL_TRY(hop_reduce(in.g, 3, in.tmp, in.r, 1.0, in.s, in.rhat, 0.0, in.sc.kappa2, WL_EVEN, 1, in.sc.state,
                      in.sc.partials, 0, site_blocks(geo), s));
    // omega = 0, so the BiCGstab p update reduces to p = z + beta p
    WL_TRY(blas_p_update(geo, in.s, in.p, in.p, in.sc.state, s));
    return WL_OK;
}

// Enqueue one BiCGstab iteration for every rhs.  ev (optional) is a pair of
// events recorded around the first hop for live kernel timing.
static int inner_iteration(Inner &in, int rhs_block, cudaStream_t s, cudaEvent_t *ev = nullptr)
{
    const Geom &geo = in.g->lat->geom;
    const int nsb = site_blocks(geo);
    const int *skip = &in.sc.state[0].done;
    const int ss = sizeof(BiState) / sizeof(int);
    const double *k2 = in.sc.kappa2;  // -kappa^2, set per mass before the graph runs
    // Under stream capture a plain cudaEventRecord only orders work inside
    // the capture; cudaEventRecordExternal (legal only while capturing)
    // makes it a real record node.
    unsigned evflags = cudaEventRecordDefault;
    if (ev) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        WL_CUDA_TRY(cudaStreamIsCapturing(s, &cs));
        if (cs == cudaStreamCaptureStatusActive) evflags = cudaEventRecordExternal;
        WL_CUDA_TRY(cudaEventRecordWithFlags(ev[0], s, evflags));
    }
    WL_TRY(hop_ex(in.g, in.p, in.tmp, nullptr, 0.0, nullptr, 0.0, 1.0, WL_ODD, 0, rhs_block, skip, ss, s));
    if (ev) WL_CUDA_TRY(cudaEventRecordWithFlags(ev[1], s, evflags));
    WL_TRY(hop_reduce(in.g, 0, in.tmp, in.p, 1.0, in.v, in.rhat, 0.0, k2, WL_EVEN, 0, in.sc.state, in.sc.partials,
                      0, nsb, s));
    WL_TRY(blas_s_update(geo, in.r, in.v, in.s, in.sc.state, s));
    WL_TRY(hop_ex(in.g, in.s, in.tmp, nullptr, 0.0, nullptr, 0.0, 1.0, WL_ODD, 0, rhs_block, skip, ss, s));
    WL_TRY(hop_reduce(in.g, 1, in.tmp, in.s, 1.0, in.t, in.rhat, 0.0, k2, WL_EVEN, 0, in.sc.state, in.sc.partials,
                      0, nsb, s));
    WL_TRY(blas_xr_update(geo, in.e, in.p, in.s, in.t, in.r, in.rhat, in.sc.state, in.sc.partials, s));
    WL_TRY(blas_p_update(geo, in.r, in.p, in.v, in.sc.state, s));
    return WL_OK;
}

// Enqueue one iteration of CG on the normal equations M^dag M e = M^dag r
// (M = M_prec, M^dag = gamma5 M gamma5, the dagger hops):
//   w = M p (||w||^2 -> alpha = ||z||^2 / ||w||^2);  e += alpha p;
//   r -= alpha w (||r||^2: stop on the true inner residual);
//   z = M^dag r (||z||^2 -> beta);  p = z + beta p.
// Buffers: v holds w, s holds z.
static int inner_iteration_cg(Inner &in, int rhs_block, cudaStream_t s, cudaEvent_t *ev = nullptr)
{
    const Geom &geo = in.g->lat->geom;
    const int nsb = site_blocks(geo);
    const int *skip = &in.sc.state[0].done;
    const int ss = sizeof(BiState) / sizeof(int);
    const double *k2 = in.sc.kappa2;
    unsigned evflags = cudaEventRecordDefault;
    if (ev) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        WL_CUDA_TRY(cudaStreamIsCapturing(s, &cs));
        if (cs == cudaStreamCaptureStatusActive) evflags = cudaEventRecordExternal;
        WL_CUDA_TRY(cudaEventRecordWithFlags(ev[0], s, evflags));
    }
    WL_TRY(hop_ex(in.g, in.p, in.tmp, nullptr, 0.0, nullptr, 0.0, 1.0, WL_ODD, 0, rhs_block, skip, ss, s));
    if (ev) WL_CUDA_TRY(cudaEventRecordWithFlags(ev[1], s, evflags));
    WL_TRY(hop_reduce(in.g, 2, in.tmp, in.p, 1.0, in.v, in.rhat, 0.0, k2, WL_EVEN, 0, in.sc.state, in.sc.partials,
                      0, nsb, s));
    WL_TRY(blas_cg_xr(geo, in.e, in.p, in.v, in.r, in.sc.state, in.sc.partials, s));
    WL_TRY(cg_normal_residual(in, rhs_block, s));
    return WL_OK;
}

// Run inner iterations until every rhs is done or max_iter is reached.
// Returns the state array copied to host in host_state.
static int run_inner(Inner &in, const wl_solver_params &prm, int max_iter, std::vector<BiState> &host_state,
                     cudaStream_t s)
{
    const int nrhs = in.nrhs;
    const int rb = prm.rhs_block;  // 0: the autotuned hop variant
    void *pin = nullptr;
    WL_TRY(in.g->pinned.get("inner_state", sizeof(BiState) * nrhs, &pin));
    BiState *hs = static_cast<BiState *>(pin);
    host_state.resize(nrhs);
    if (prm.mode == WL_MODE_PERSISTENT) {
        // one cooperative launch for all iterations; 1 s bound on every barrier wait
        WL_TRY(persistent_inner(in.g, in.prec, nrhs, in.r, in.rhat, in.p, in.v, in.s, in.t, in.tmp, in.e, in.sc.state,
                                in.sc.kappa2, max_iter, 1.0, 0, s));
        WL_CUDA_TRY(cudaMemcpyAsync(hs, in.sc.state, sizeof(BiState) * nrhs, cudaMemcpyDeviceToHost, s));
        WL_CUDA_TRY(cudaStreamSynchronize(s));
        std::memcpy(host_state.data(), hs, sizeof(BiState) * nrhs);
        return WL_OK;
    }
    const int K = prm.mode == WL_MODE_GRAPH ? std::max(1, prm.graph_iters) : 1;
    cudaGraphExec_t exec = nullptr;
    int status = WL_OK;
    // live timing of the first hop of each iteration (wl_profile_enable)
    const bool prof = in.g->profiling != 0;
    std::vector<cudaEvent_t> host_ev;   // host mode: one pair
    std::vector<int> it_before(nrhs, 0);
    long long graph_kernels = 0;
    cudaEvent_t *ev = nullptr;
    if (prm.mode == WL_MODE_GRAPH) {
        // Reuse the captured block while buffers and shape are unchanged.
        GraphCache &gc = in.g->inner_graph;
        std::vector<uintptr_t> key = {
            (uintptr_t)in.p.ptr, (uintptr_t)in.tmp.ptr, (uintptr_t)in.v.ptr, (uintptr_t)in.r.ptr,
            (uintptr_t)in.rhat.ptr, (uintptr_t)in.s.ptr, (uintptr_t)in.t.ptr, (uintptr_t)in.e.ptr,
            (uintptr_t)in.sc.state, (uintptr_t)in.sc.partials, (uintptr_t)in.sc.kappa2, (uintptr_t)nrhs,
            (uintptr_t)in.prec, (uintptr_t)in.xprec, (uintptr_t)K, (uintptr_t)rb, (uintptr_t)prof,
            (uintptr_t)prm.inner_solver,
            (uintptr_t)in.g->lat->geom.Vh};
        if (gc.exec == nullptr || gc.key != key) {
            gc.release();
            gc.events.resize(prof ? 2 * K : 0);
            for (auto &e : gc.events) WL_CUDA_TRY(cudaEventCreate(&e));
            cudaStream_t cap = nullptr;
            WL_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
            cudaGraph_t graph = nullptr;
            cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                for (int k = 0; k < K && status == WL_OK; ++k)
                    status = prm.inner_solver == WL_SOLVER_CG
                                 ? inner_iteration_cg(in, rb, cap, prof ? &gc.events[2 * k] : nullptr)
                                 : inner_iteration(in, rb, cap, prof ? &gc.events[2 * k] : nullptr);
                e = cudaStreamEndCapture(cap, &graph);
            }
            if (e == cudaSuccess && status == WL_OK) e = cudaGraphInstantiate(&gc.exec, graph, 0);
            if (graph) {
                // kernel nodes only (event-record nodes are not launches)
                size_t n = 0;
                cudaGraphGetNodes(graph, nullptr, &n);
                std::vector<cudaGraphNode_t> nodes(n);
                if (n) cudaGraphGetNodes(graph, nodes.data(), &n);
                gc.kernels = 0;
                for (auto nd : nodes) {
                    cudaGraphNodeType t;
                    if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++gc.kernels;
                }
                cudaGraphDestroy(graph);
            }
            cudaStreamDestroy(cap);
            if (e != cudaSuccess || status != WL_OK) {
                gc.release();
                if (status == WL_OK) {
                    set_error(std::string("graph capture: ") + cudaGetErrorString(e));
                    status = WL_ERR_CUDA;
                }
                return status;
            }
            gc.key = key;
        }
        exec = gc.exec;
        graph_kernels = gc.kernels;
        if (prof) ev = gc.events.data();
    } else if (prof) {
        host_ev.resize(2);
        for (auto &e : host_ev) WL_CUDA_TRY(cudaEventCreate(&e));
        ev = host_ev.data();
    }
    struct EvFree {
        std::vector<cudaEvent_t> &v;
        ~EvFree() { for (auto e : v) cudaEventDestroy(e); }
    } ev_free{host_ev};
    int done_iters = 0;
    for (;;) {
        if (exec) {
            cudaError_t e = cudaGraphLaunch(exec, s);
            if (e != cudaSuccess) {
                set_error(std::string("cudaGraphLaunch: ") + cudaGetErrorString(e));
                status = WL_ERR_CUDA;
                break;
            }
            add_launches(graph_kernels);
            done_iters += K;
        } else {
            status = prm.inner_solver == WL_SOLVER_CG ? inner_iteration_cg(in, rb, s, ev) : inner_iteration(in, rb, s, ev);
            if (status != WL_OK) break;
            done_iters += 1;
        }
        cudaError_t e = cudaMemcpyAsync(hs, in.sc.state, sizeof(BiState) * nrhs, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            set_error(std::string("inner loop: ") + cudaGetErrorString(e));
            status = WL_ERR_CUDA;
            break;
        }
        if (prof) {
            // iterations of this block in which every rhs ran: the smallest
            // per-rhs advance among rhs that were active
            int full = K;
            int n_act = 0;
            for (int r = 0; r < nrhs; ++r) {
                const int d = hs[r].iters - it_before[r];
                if (d > 0 || !hs[r].done) { full = std::min(full, d); ++n_act; }
                it_before[r] = hs[r].iters;
            }
            wl_kernel_profile &P = in.g->prof[prec_index(in.prec)];
            const double vh = (double)in.g->lat->geom.Vh;
            for (int k = 0; k < full && n_act == nrhs; ++k) {
                float ms = 0.f;
                if (cudaEventElapsedTime(&ms, ev[2 * k], ev[2 * k + 1]) == cudaSuccess) {
                    P.launches += 1;
                    P.ms += ms;
                    P.site_rhs += vh * nrhs;
                    P.sites += vh;
                } else {
                    (void)cudaGetLastError();  // not recorded: skip, and keep the error state clean
                }
            }
        }
        bool all = true;
        for (int r = 0; r < nrhs; ++r) all &= hs[r].done != 0;
        if (all || done_iters >= max_iter) break;
    }
    std::memcpy(host_state.data(), hs, sizeof(BiState) * nrhs);
    if (status == WL_OK && hop_variant_for(in.g, in.prec, nrhs, rb) >= 9000) {
        // a TMA-staged hop that stopped waiting leaves its tile unwritten
        unsigned faults = 0;
        WL_TRY(wait_faults(&faults, true, s));
        if (faults) {
            set_error("inner solve: a TMA-staged hop gave up waiting for its copies");
            return WL_ERR_TIMEOUT;
        }
    }
    return status;
}

// ----------------------------------------------------- outer (FP64) loop

struct Timer {
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    double sec() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

static double default_inner_tol(int prec)
{
    return prec == WL_F32 ? 1e-6 : prec == WL_F16 ? 3e-4 : 1e-12;
}

// Solve M_prec x = bprec for nrhs right-hand sides by defect correction:
//   r = bprec - M_prec x (FP64); stop when ||r|| <= tol * bnorm;
//   inner BiCGstab in prec on M_prec e = r to relative residual delta;
//   x += e (FP64).
// x64 holds the initial guesses and receives the solutions.
// y_out (optional) receives D_eo D_oe x of each rhs's final x, so later masses
// can form their first residual by linear combination.  With r0_given the
// caller has already put b_prec - M_prec x into dc_r64: the first check
// uses it without hops; it never declares convergence by itself (that needs
// a hop-based check, which also produces D_oe x for the reconstruction).
// rn2_out (optional) receives ||b_prec - M_prec x||^2 of each rhs's final x
// from its last hop-based check.
static int eo_defect_correction(wl_gauge *g, const Vec &bprec, const Vec &x64, double kappa,
                                const wl_solver_params &prm, const std::vector<double> &bnorm,
                                std::vector<wl_solver_stats> &stats, cudaStream_t s, const Vec *y_out = nullptr,
                                bool r0_given = false, std::vector<double> *rn2_out = nullptr)
{
    const Geom &geo = g->lat->geom;
    const int nrhs = bprec.nrhs;
    const int prec = prm.inner_prec;
    Inner in;
    WL_TRY(make_inner(g, prec, nrhs, kappa, &in, s));
    if (prm.rhs_block == 0) {  // tune before any graph capture
        WL_TRY(autotune_hop(g, prec, nrhs, s, nullptr));
        WL_TRY(autotune_hop(g, x64.prec, nrhs, s, nullptr));
    }
    Vec r64, tmp64;  // outer precision (FP64 or double-float)
    WL_TRY(make_vec(g, "dc_r64", x64.prec, nrhs, &r64));
    WL_TRY(make_vec(g, "dc_tmp64", x64.prec, nrhs, &tmp64));
    void *pin = nullptr;
    WL_TRY(g->pinned.get("dc_scalars", nrhs * (sizeof(double) * 2 + sizeof(int) * 2), &pin));
    double *h_rn2 = static_cast<double *>(pin);
    double *h_delta2 = h_rn2 + nrhs;
    int *h_active = reinterpret_cast<int *>(h_delta2 + nrhs);
    int *h_outer = h_active + nrhs;
    const double delta0 = prm.inner_tol > 0 ? prm.inner_tol : default_inner_tol(prec);
    std::vector<int> outer_done(nrhs, 0), iters(nrhs, 0), restarts(nrhs, 0), fails(nrhs, 0);
    // reliable updates: an inner run that converged can be continued (mode 2)
    std::vector<int> can_continue(nrhs, 0);
    std::vector<double> last_rn(nrhs, INFINITY);
    std::vector<BiState> hst;
    const double k2 = kappa * kappa;
    const double mk2 = -k2;
    WL_CUDA_TRY(cudaMemcpyAsync(in.sc.kappa2, &mk2, sizeof(double), cudaMemcpyHostToDevice, s));
    WL_CUDA_TRY(cudaMemsetAsync(in.sc.outer_done, 0, sizeof(int) * nrhs, s));
    int total_restarts = 0;
    bool lincomb_check = r0_given;
    // outer residual hops: autotuned full grid, or the FP64 grid-stride form
    const int ohop = (prm.outer_blocks_per_sm > 0 && x64.prec == WL_F64)
                         ? -(7000 + 100 * (nrhs >= 2 ? 2 : 1) + prm.outer_blocks_per_sm)
                         : 0;
    // Three levels for FP16 inner solves (prm.inner_refine): an FP16 BiCGstab
    // stops near 3e-4 of its starting residual, where the FP16 rounding of its
    // first iterations leaves the true residual; so one outer step runs FP16
    // segments, recomputes the inner residual r_in - M e in FP32 between them
    // (e is the FP32 accumulator, kept across segments) and stops at
    // refine_tol (1e-7 by default, near what an FP32 recomputation and an
    // FP32 accumulator allow; segments that stop halving the residual end
    // earlier) of the outer residual.  The FP64 check that follows then
    // gains 1e-6 to 1e-7 instead of 3e-4.
    const bool refine = prm.inner_refine && prec == WL_F16 && !prm.reliable &&
                        prm.inner_solver == WL_SOLVER_BICGSTAB && (g->prec_mask & WL_F32);
    Vec rin32, r32, tmp32;
    int *mid_skip = nullptr;
    double *h_rn32 = nullptr, *h_mdelta2 = nullptr;
    int *h_mode = nullptr, *h_skip = nullptr;
    if (refine) {
        WL_TRY(make_vec(g, "dc_rin32", WL_F32, nrhs, &rin32));
        WL_TRY(make_vec(g, "dc_r32", WL_F32, nrhs, &r32));
        WL_TRY(make_vec(g, "dc_tmp32", WL_F32, nrhs, &tmp32));
        void *pp = nullptr;
        WL_TRY(g->ws.get("dc_mid_skip", sizeof(int) * nrhs, &pp));
        mid_skip = static_cast<int *>(pp);
        if (prm.rhs_block == 0) WL_TRY(autotune_hop(g, WL_F32, nrhs, s, nullptr));
        void *pin2 = nullptr;
        WL_TRY(g->pinned.get("dc_mid", nrhs * (sizeof(double) * 2 + sizeof(int) * 2), &pin2));
        h_rn32 = static_cast<double *>(pin2);
        h_mdelta2 = h_rn32 + nrhs;
        h_mode = reinterpret_cast<int *>(h_mdelta2 + nrhs);
        h_skip = h_mode + nrhs;
    }
    const double refine_tol = prm.inner_tol > 0 ? prm.inner_tol : 1e-7;
    std::vector<double> d_outer(nrhs, 0.0), rn_outer(nrhs, 0.0);
    // live timing of the first residual hop of every check (wl_profile_enable)
    struct Ev {
        cudaEvent_t e[2] = {nullptr, nullptr};
        ~Ev() { for (auto x : e) if (x) cudaEventDestroy(x); }
    } ev;
    if (g->profiling)
        for (auto &x : ev.e) WL_CUDA_TRY(cudaEventCreate(&x));
    for (;;) {
        // r = bprec - x + kappa^2 D_eo D_oe x for the rhs still iterating;
        // D_oe x stays in tmp64 (the reconstruction uses the last one)
        int n_hop = 0;  // rhs the residual hops process
        if (!lincomb_check) {
            for (int r = 0; r < nrhs; ++r) n_hop += outer_done[r] ? 0 : 1;
            if (ev.e[0]) WL_CUDA_TRY(cudaEventRecord(ev.e[0], s));
            WL_TRY(hop_ex(g, x64, tmp64, nullptr, 0.0, nullptr, 0.0, 1.0, WL_ODD, 0, ohop, in.sc.outer_done, 1, s));
            if (ev.e[1]) WL_CUDA_TRY(cudaEventRecord(ev.e[1], s));
            WL_TRY(hop_ex(g, tmp64, r64, &bprec, 1.0, &x64, -1.0, k2, WL_EVEN, 0, ohop, in.sc.outer_done, 1, s,
                          y_out));
        }
        WL_TRY(blas_norm2(geo, r64, in.sc.norms, in.sc.partials, in.sc.tickets, s));
        WL_CUDA_TRY(cudaMemcpyAsync(h_rn2, in.sc.norms, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s));
        WL_CUDA_TRY(cudaStreamSynchronize(s));
        if (ev.e[0] && n_hop > 0) {
            float ms = 0.f;
            WL_CUDA_TRY(cudaEventElapsedTime(&ms, ev.e[0], ev.e[1]));
            wl_kernel_profile &P = g->prof[3];
            P.launches += 1;
            P.ms += ms;
            P.site_rhs += (double)geo.Vh * n_hop;
            P.sites += (double)geo.Vh;
        }
        int n_active = 0;
        for (int r = 0; r < nrhs; ++r) {
            const double rn = std::sqrt(h_rn2[r]);
            h_active[r] = 0;
            if (outer_done[r]) continue;
            if (!std::isfinite(rn)) {
                outer_done[r] = 1;
                stats[r].status = WL_ERR_BREAKDOWN;
                set_error("defect correction: non-finite true residual (rhs " + std::to_string(r) + ")");
                continue;
            }
            if (rn <= prm.tol * bnorm[r]) {
                if (lincomb_check) continue;  // confirmed by the next, hop-based check
                outer_done[r] = 1;
                stats[r].status = WL_OK;
                continue;
            }
            if (iters[r] >= prm.max_iter || restarts[r] >= prm.max_restarts || fails[r] >= 5) {
                outer_done[r] = 1;
                stats[r].status = fails[r] >= 5 ? WL_ERR_BREAKDOWN : WL_ERR_NOCONV;
                set_error(std::string("defect correction: ") +
                          (fails[r] >= 5 ? "five restarts without halving the residual"
                                         : "iteration or restart cap reached") +
                          " (rhs " + std::to_string(r) + ")");
                continue;
            }
            // no need to iterate the inner solve below what the outer target needs
            const double need = 0.5 * prm.tol * bnorm[r] / rn;
            const double d = std::max(delta0, need);
            h_delta2[r] = d * d;
            if (refine) {
                // the outer step aims at refine_tol; its first FP16 segment at
                // the FP16 tolerance
                d_outer[r] = std::max(refine_tol, need);
                rn_outer[r] = rn;
                const double d16 = std::max(default_inner_tol(WL_F16), d_outer[r]);
                h_delta2[r] = d16 * d16;
            }
            h_active[r] = (prm.reliable && can_continue[r]) ? 2 : 1;
            fails[r] = rn >= 0.5 * last_rn[r] ? fails[r] + 1 : 0;  // stagnation guard
            last_rn[r] = rn;
            ++n_active;
        }
        for (int r = 0; r < nrhs; ++r) h_outer[r] = outer_done[r];
        WL_CUDA_TRY(cudaMemcpyAsync(in.sc.outer_done, h_outer, sizeof(int) * nrhs, cudaMemcpyHostToDevice, s));
        const bool was_lincomb = lincomb_check;
        lincomb_check = false;
        if (n_active == 0) {
            if (was_lincomb) continue;  // every guess already good: confirm with hops
            break;
        }
        WL_CUDA_TRY(cudaMemcpyAsync(in.sc.active, h_active, sizeof(int) * nrhs, cudaMemcpyHostToDevice, s));
        WL_CUDA_TRY(cudaMemcpyAsync(in.sc.delta2, h_delta2, sizeof(double) * nrhs, cudaMemcpyHostToDevice, s));
        WL_TRY(blas_restart(geo, r64, in.r, in.rhat, in.p, in.e, in.sc.state, in.sc.partials, in.sc.active,
                            in.sc.delta2, s));
        if (prm.inner_solver == WL_SOLVER_CG) WL_TRY(cg_normal_residual(in, 0, s));  // z = M^dag r, p = z
        bool any_continue = false;
        for (int r = 0; r < nrhs; ++r) any_continue |= h_active[r] == 2;
        // continued rhs: p = r + beta (p - omega v) with the beta the update set
        // (restarted rhs have beta = omega = 0, so p = r stays)
        if (any_continue) WL_TRY(blas_p_update(geo, in.r, in.p, in.v, in.sc.state, s));
        int cap = 0;
        for (int r = 0; r < nrhs; ++r)
            if (h_active[r]) cap = std::max(cap, prm.max_iter - iters[r]);
        WL_TRY(run_inner(in, prm, cap, hst, s));
        for (int r = 0; r < nrhs; ++r)
            if (h_active[r]) iters[r] += hst[r].iters;
        // Further segments only for the rhs whose outer target lies below
        // what one FP16 solve reaches: for the others the first segment
        // already aimed at the target, and the FP64 check verifies it.
        std::vector<int> mid(nrhs, 0);
        int n_seg = 0;
        if (refine)
            for (int r = 0; r < nrhs; ++r) {
                mid[r] = h_active[r] != 0 && d_outer[r] < default_inner_tol(WL_F16);
                n_seg += mid[r];
            }
        if (n_seg > 0) {
            // FP32 copy of this outer step's right-hand side, then segments
            WL_TRY(blas_convert(geo, r64, rin32, s));
            std::vector<double> seg_start(nrhs, 0.0);
            for (int r = 0; r < nrhs; ++r) seg_start[r] = rn_outer[r];
            const int kMaxSegments = 8;
            for (int seg = 1;; ++seg) {
                // r32 = r_in - M_prec e in FP32 for the rhs still segmenting
                for (int r = 0; r < nrhs; ++r) h_skip[r] = mid[r] ? 0 : 1;
                WL_CUDA_TRY(cudaMemcpyAsync(mid_skip, h_skip, sizeof(int) * nrhs, cudaMemcpyHostToDevice, s));
                WL_TRY(hop_ex(g, in.e, tmp32, nullptr, 0.0, nullptr, 0.0, 1.0, WL_ODD, 0, 0, mid_skip, 1, s));
                WL_TRY(hop_ex(g, tmp32, r32, &rin32, 1.0, &in.e, -1.0, k2, WL_EVEN, 0, 0, mid_skip, 1, s));
                WL_TRY(blas_norm2(geo, r32, in.sc.norms, in.sc.partials, in.sc.tickets, s));
                WL_CUDA_TRY(cudaMemcpyAsync(h_rn32, in.sc.norms, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s));
                WL_CUDA_TRY(cudaStreamSynchronize(s));
                int n_mid = 0;
                for (int r = 0; r < nrhs; ++r) {
                    h_mode[r] = 0;
                    if (!mid[r]) continue;
                    const double rn32 = std::sqrt(h_rn32[r]);
                    // done: at the outer step's target, no longer halving,
                    // broken down, out of segments or iterations
                    if (!(rn32 > d_outer[r] * rn_outer[r]) || !std::isfinite(rn32) || rn32 > 0.5 * seg_start[r] ||
                        hst[r].breakdown || seg >= kMaxSegments || iters[r] >= prm.max_iter) {
                        mid[r] = 0;
                        continue;
                    }
                    const double d16 = std::max(default_inner_tol(WL_F16), 0.5 * d_outer[r] * rn_outer[r] / rn32);
                    h_mdelta2[r] = d16 * d16;
                    h_mode[r] = 3;   // restart from r32, keeping e
                    seg_start[r] = rn32;
                    ++n_mid;
                }
                if (n_mid == 0) break;
                WL_CUDA_TRY(cudaMemcpyAsync(in.sc.active, h_mode, sizeof(int) * nrhs, cudaMemcpyHostToDevice, s));
                WL_CUDA_TRY(cudaMemcpyAsync(in.sc.delta2, h_mdelta2, sizeof(double) * nrhs, cudaMemcpyHostToDevice, s));
                WL_TRY(blas_restart(geo, r32, in.r, in.rhat, in.p, in.e, in.sc.state, in.sc.partials, in.sc.active,
                                    in.sc.delta2, s));
                int mcap = 0;
                for (int r = 0; r < nrhs; ++r)
                    if (h_mode[r]) mcap = std::max(mcap, prm.max_iter - iters[r]);
                WL_TRY(run_inner(in, prm, mcap, hst, s));
                for (int r = 0; r < nrhs; ++r)
                    if (h_mode[r]) iters[r] += hst[r].iters;
            }
            // the outer step's active set for the accumulation
            WL_CUDA_TRY(cudaMemcpyAsync(in.sc.active, h_active, sizeof(int) * nrhs, cudaMemcpyHostToDevice, s));
        }
        WL_TRY(blas_accum(geo, in.e, x64, in.sc.active, s));
        for (int r = 0; r < nrhs; ++r)
            if (h_active[r]) {
                restarts[r] += 1;
                can_continue[r] = hst[r].done && !hst[r].breakdown && hst[r].iters > 0;
            }
        ++total_restarts;
    }
    for (int r = 0; r < nrhs; ++r) {
        stats[r].iterations = iters[r];
        stats[r].matvecs = 2 * iters[r] + restarts[r] + 1;
        stats[r].restarts = restarts[r];
    }
    if (rn2_out) rn2_out->assign(h_rn2, h_rn2 + nrhs);
    (void)total_restarts;
    return WL_OK;
}

// Per-rhs FP64 squared norms of one parity vector (host result).
static int norms2_host(wl_gauge *g, const Vec &v, Scratch &sc, std::vector<double> &out, cudaStream_t s)
{
    const int n = v.nrhs;
    WL_TRY(blas_norm2(g->lat->geom, v, sc.norms, sc.partials, sc.tickets, s));
    out.resize(n);
    WL_CUDA_TRY(cudaMemcpyAsync(out.data(), sc.norms, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    WL_CUDA_TRY(cudaStreamSynchronize(s));
    return WL_OK;
}

// FP64 relative residuals ||b - M_k x|| / ||b|| over the full lattice for
// nrhs vectors given by their halves.
int full_relres(wl_gauge *g, const Vec &be, const Vec &bo, const Vec &xe, const Vec &xo, double kappa,
                const std::vector<double> &bnorm, std::vector<double> &relres, cudaStream_t s,
                const std::vector<double> *ro_norm2)
{
    const int nrhs = be.nrhs;
    Vec re, ro;
    WL_TRY(make_vec(g, "rr_re", be.prec, nrhs, &re));
    // r_e = b_e - x_e + kappa D_eo x_o ; r_o = b_o - x_o + kappa D_oe x_e
    WL_TRY(hop_ex(g, xo, re, &be, 1.0, &xe, -1.0, kappa, WL_EVEN, 0, 0, nullptr, 0, s));
    Scratch sc;
    WL_TRY(get_scratch(g, nrhs, &sc, s));
    std::vector<double> n2e, n2o;
    WL_TRY(norms2_host(g, re, sc, n2e, s));
    if (ro_norm2) {
        n2o = *ro_norm2;
    } else {
        WL_TRY(make_vec(g, "rr_ro", be.prec, nrhs, &ro));
        WL_TRY(hop_ex(g, xe, ro, &bo, 1.0, &xo, -1.0, kappa, WL_ODD, 0, 1, nullptr, 0, s));
        WL_TRY(norms2_host(g, ro, sc, n2o, s));
    }
    relres.resize(nrhs);
    for (int r = 0; r < nrhs; ++r) relres[r] = bnorm[r] > 0 ? std::sqrt(n2e[r] + n2o[r]) / bnorm[r] : 0.0;
    return WL_OK;
}

// Exports of finished masses on a side stream, overlapped with the solve of
// the next mass (the canonical solutions may be page-locked host memory,
// written at the host link's rate).  The side stream has the highest
// priority and the export a grid of one looping block per SM, so it starts
// as soon as a few SM slots free up and then streams on them while the
// solver's kernels fill the rest.  The odd halves x_o alternate between
// two buffers; a mass waits for the export of the mass two before it ahead
// of overwriting one.  Destruction waits for every export.
struct AsyncExport {
    cudaStream_t stream = nullptr;
    cudaEvent_t ready[2] = {nullptr, nullptr}, done[2] = {nullptr, nullptr};
    bool pending[2] = {false, false};
    int slot = 0;
    // Export grid.  Into device memory: the SM count.  Into page-locked host
    // memory, where the host link bounds the export, a tenth of it: the few
    // blocks still keep the link busy and leave the other SMs to the next
    // mass's solve (48^3x96, 12 sources x 16 masses, end to end: 7.98 s with
    // 16 blocks against 8.76 s with 152; the device-memory export needs the
    // full grid).
    int blocks = 0;
    int full_blocks = 0;   // the SM count: the last mass's export runs alone
    int init()
    {
        int dev = 0;
        WL_CUDA_TRY(cudaGetDevice(&dev));
        WL_CUDA_TRY(cudaDeviceGetAttribute(&blocks, cudaDevAttrMultiProcessorCount, dev));
        full_blocks = blocks;
        int lo = 0, hi = 0;
        WL_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&lo, &hi));
        WL_CUDA_TRY(cudaStreamCreateWithPriority(&stream, cudaStreamNonBlocking, hi));
        for (int k = 0; k < 2; ++k) {
            WL_CUDA_TRY(cudaEventCreateWithFlags(&ready[k], cudaEventDisableTiming));
            WL_CUDA_TRY(cudaEventCreateWithFlags(&done[k], cudaEventDisableTiming));
        }
        return WL_OK;
    }
    // order everything after the last export on s
    int join(cudaStream_t s)
    {
        for (int k = 0; k < 2; ++k)
            if (pending[k]) WL_CUDA_TRY(cudaStreamWaitEvent(s, done[k], 0));
        return WL_OK;
    }
    ~AsyncExport()
    {
        if (stream) cudaStreamSynchronize(stream);
        for (int k = 0; k < 2; ++k) {
            if (ready[k]) cudaEventDestroy(ready[k]);
            if (done[k]) cudaEventDestroy(done[k]);
        }
        if (stream) cudaStreamDestroy(stream);
    }
};

// One mass for nrhs sources already imported as be, bo (outer precision),
// with bprec = b_e + kappa D_eo b_o prepared by the caller: solve, rebuild
// x_o = b_o + kappa D_oe x_e, compute the full-lattice residual, export x
// (on s, or on the side stream of ax).
//
// Full-lattice residual (Section 6.2.3).  With x_o rebuilt from the D_oe x_e
// of the last check, r_o = b_o - x_o + kappa D_oe x_e is the rounding of that
// rebuild (the reconstruction pass returns its norm) and
//   r_e = b_e - x_e + kappa D_eo x_o = b_prec - M_prec x_e + kappa D_eo (x_o - b_o - kappa D_oe x_e),
// i.e. the preconditioned residual of the last check plus kappa D_eo applied
// to that rounding, below 1e-15 of ||x||.  So ||r||^2 = ||r_prec||^2 + ||r_o||^2
// needs no further hop; prm.verify_full recomputes r_e with one more hop
// D_eo x_o instead.
static int solve_one_mass(wl_gauge *g, const Vec &be, const Vec &bo, const Vec &bprec, const Vec &xe, double m0,
                          const wl_solver_params &prm, const std::vector<double> &bnorm2, void *const *x_out,
                          int x_out_stride, std::vector<wl_solver_stats> &stats, cudaStream_t s,
                          const Vec *y_out = nullptr, bool r0_given = false, AsyncExport *ax = nullptr)
{
    const Geom &geo = g->lat->geom;
    const int nrhs = be.nrhs;
    const double kappa = 1.0 / (2.0 * m0 + 8.0);
    const int slot = ax ? ax->slot : 0;
    Vec xo;
    WL_TRY(make_vec(g, ax ? (slot ? "mm_xo1" : "mm_xo0") : "mm_xo", xe.prec, nrhs, &xo));
    std::vector<double> bnorm(nrhs);
    for (int r = 0; r < nrhs; ++r) bnorm[r] = std::sqrt(bnorm2[r]);
    std::vector<double> rn2;
    WL_TRY(eo_defect_correction(g, bprec, xe, kappa, prm, bnorm, stats, s, y_out, r0_given, &rn2));
    // The last residual check left D_oe x_e (final x_e) in dc_tmp64:
    // x_o = b_o + kappa D_oe x_e and the odd residual in one vector pass.
    Vec dx;
    WL_TRY(make_vec(g, "dc_tmp64", xe.prec, nrhs, &dx));
    Scratch sc;
    WL_TRY(get_scratch(g, nrhs, &sc, s));
    if (ax && ax->pending[slot]) WL_CUDA_TRY(cudaStreamWaitEvent(s, ax->done[slot], 0));
    WL_TRY(blas_recon(geo, bo, dx, kappa, xo, sc.norms, sc.partials, sc.tickets, s));
    std::vector<double> ro2(nrhs);
    WL_CUDA_TRY(cudaMemcpyAsync(ro2.data(), sc.norms, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s));
    WL_CUDA_TRY(cudaStreamSynchronize(s));
    std::vector<double> rel(nrhs);
    if (prm.verify_full) {
        WL_TRY(full_relres(g, be, bo, xe, xo, kappa, bnorm, rel, s, &ro2));
    } else {
        for (int r = 0; r < nrhs; ++r) rel[r] = bnorm[r] > 0 ? std::sqrt(rn2[r] + ro2[r]) / bnorm[r] : 0.0;
    }
    std::vector<void *> outs(nrhs);
    for (int r = 0; r < nrhs; ++r) {
        stats[r].mass = m0;
        stats[r].true_relres = rel[r];
        outs[r] = x_out[(size_t)r * x_out_stride];
    }
    if (!ax) return export_full(geo, xe, xo, outs.data(), s);
    WL_CUDA_TRY(cudaEventRecord(ax->ready[slot], s));
    WL_CUDA_TRY(cudaStreamWaitEvent(ax->stream, ax->ready[slot], 0));
    WL_TRY(export_full(geo, xe, xo, outs.data(), ax->stream, ax->blocks));
    WL_CUDA_TRY(cudaEventRecord(ax->done[slot], ax->stream));
    ax->pending[slot] = true;
    ax->slot ^= 1;
    return WL_OK;
}

static int check_params(const wl_gauge *g, const wl_solver_params *p)
{
    if (!p || !(p->tol > 0) || p->max_iter < 1 || !valid_prec(p->inner_prec) || p->inner_prec == WL_DF ||
        p->max_restarts < 1 || (p->mode != WL_MODE_HOST && p->mode != WL_MODE_GRAPH && p->mode != WL_MODE_PERSISTENT) ||
        p->graph_iters < 0 || p->guess < WL_GUESS_ZERO || p->guess > WL_GUESS_SSM || p->guess_max < 0 ||
        (p->reliable != 0 && p->reliable != 1) ||
        (p->inner_solver != WL_SOLVER_BICGSTAB && p->inner_solver != WL_SOLVER_CG) ||
        (p->inner_solver == WL_SOLVER_CG && (p->reliable || p->mode == WL_MODE_PERSISTENT)) ||
        p->rhs_block < 0 || p->rhs_block > 4 || (p->outer_prec != WL_F64 && p->outer_prec != WL_DF) ||
        (p->verify_full != 0 && p->verify_full != 1) || p->outer_blocks_per_sm < 0 || p->outer_blocks_per_sm > 2 ||
        (p->inner_refine != 0 && p->inner_refine != 1)) {
        set_error("solver parameters out of range");
        return WL_ERR_ARG;
    }
    if (!(g->prec_mask & p->outer_prec) || !(g->prec_mask & p->inner_prec)) {
        set_error("gauge handle needs links of the outer and of the inner precision");
        return WL_ERR_ARG;
    }
    if (p->inner_refine && p->inner_prec == WL_F16 && !(g->prec_mask & WL_F32)) {
        set_error("inner_refine with an FP16 inner solve needs FP32 links on the gauge handle");
        return WL_ERR_ARG;
    }
    return WL_OK;
}

}  // namespace wl

using namespace wl;

// ---------------------------------------------------------------- C ABI

extern "C" int wl_persistent_selftest(wl_gauge *g, int prec, int inject_missing_arrival, double wait_limit_s,
                                      void *stream)
{
    if (!g || (prec != WL_F32 && prec != WL_F16 && prec != WL_F64) || !(g->prec_mask & prec) ||
        !(wait_limit_s > 0.0) || wait_limit_s > 10.0) {
        set_error("wl_persistent_selftest: bad argument");
        return WL_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g->mu);
    cudaStream_t s = as_stream(stream);
    Inner in;
    WL_TRY(make_inner(g, prec, 1, 0.1, &in, s));
    const size_t b = in.r.rhs_bytes;
    for (Vec *v : {&in.r, &in.rhat, &in.p, &in.v, &in.s, &in.t, &in.tmp}) WL_CUDA_TRY(cudaMemsetAsync(v->ptr, 0, b, s));
    WL_CUDA_TRY(cudaMemsetAsync(in.e.ptr, 0, in.e.rhs_bytes, s));
    // one live rhs with a large target so the loop runs its iterations
    BiState st;
    std::memset(&st, 0, sizeof(st));
    st.rho_re = 1.0;
    st.target2 = -1.0;
    WL_CUDA_TRY(cudaMemcpyAsync(in.sc.state, &st, sizeof(st), cudaMemcpyHostToDevice, s));
    const double mk2 = -0.01;
    WL_CUDA_TRY(cudaMemcpyAsync(in.sc.kappa2, &mk2, sizeof(double), cudaMemcpyHostToDevice, s));
    return persistent_inner(g, prec, 1, in.r, in.rhat, in.p, in.v, in.s, in.t, in.tmp, in.e, in.sc.state, in.sc.kappa2,
                            2, wait_limit_s, inject_missing_arrival ? 1 : 0, s);
}

extern "C" int wl_vector_op(wl_gauge *g, int kind, int prec, int n_rhs, size_t rhs_stride, void *const *vecs,
                            const double *scal, double *dots, void *stream)
{
    const int nv = kind == WL_VEC_S ? 3 : kind == WL_VEC_XR ? 6 : kind == WL_VEC_P ? 3 : kind == WL_VEC_NORM2 ? 1 : 0;
    if (!g || nv == 0 || !vecs || n_rhs < 1 || n_rhs > 64 || !valid_prec(prec) || prec == WL_DF ||
        (kind != WL_VEC_NORM2 && !scal) || ((kind == WL_VEC_XR || kind == WL_VEC_NORM2) && !dots)) {
        set_error("wl_vector_op: bad argument");
        return WL_ERR_ARG;
    }
    const Geom &geo = g->lat->geom;
    const size_t need = (spinor_bytes(geo, prec) + 255) & ~(size_t)255;
    const size_t need_x = (spinor_bytes(geo, prec == WL_F64 ? WL_F64 : WL_F32) + 255) & ~(size_t)255;
    if (rhs_stride < std::max(need, kind == WL_VEC_XR ? need_x : need) || rhs_stride % 256) {
        set_error("wl_vector_op: rhs_stride must be a multiple of 256 holding one internal vector");
        return WL_ERR_ARG;
    }
    for (int k = 0; k < nv; ++k)
        if (!vecs[k]) { set_error("wl_vector_op: NULL vector"); return WL_ERR_ARG; }
    std::lock_guard<std::mutex> lock(g->mu);
    cudaStream_t s = as_stream(stream);
    Vec v[6];
    for (int k = 0; k < nv; ++k) {
        v[k].ptr = vecs[k];
        v[k].prec = prec;
        v[k].nrhs = n_rhs;
        v[k].rhs_bytes = rhs_stride;
    }
    Scratch sc;
    WL_TRY(get_scratch(g, n_rhs, &sc, s));
    std::vector<BiState> hs(n_rhs);
    for (int r = 0; r < n_rhs && kind != WL_VEC_NORM2; ++r) {
        BiState &b = hs[r];
        std::memset(&b, 0, sizeof(b));
        b.alpha_re = scal[6 * r + 0];
        b.alpha_im = scal[6 * r + 1];
        b.omega_re = scal[6 * r + 2];
        b.omega_im = scal[6 * r + 3];
        b.beta_re = scal[6 * r + 4];
        b.beta_im = scal[6 * r + 5];
        b.rho_re = 1.0;       // previous <rhat, r>: lets the update evaluate beta
        b.target2 = -1.0;     // never converged
    }
    if (kind != WL_VEC_NORM2)
        WL_CUDA_TRY(cudaMemcpyAsync(sc.state, hs.data(), sizeof(BiState) * n_rhs, cudaMemcpyHostToDevice, s));
    if (kind == WL_VEC_S) {
        WL_TRY(blas_s_update(geo, v[0], v[1], v[2], sc.state, s));
    } else if (kind == WL_VEC_P) {
        WL_TRY(blas_p_update(geo, v[0], v[1], v[2], sc.state, s));
    } else if (kind == WL_VEC_XR) {
        v[0].prec = prec == WL_F64 ? WL_F64 : WL_F32;   // the accumulator of the inner solve
        WL_TRY(blas_xr_update(geo, v[0], v[1], v[2], v[3], v[4], v[5], sc.state, sc.partials, s));
        WL_CUDA_TRY(cudaMemcpyAsync(hs.data(), sc.state, sizeof(BiState) * n_rhs, cudaMemcpyDeviceToHost, s));
    } else {
        WL_TRY(blas_norm2(geo, v[0], sc.norms, sc.partials, sc.tickets, s));
        WL_CUDA_TRY(cudaMemcpyAsync(dots, sc.norms, sizeof(double) * n_rhs, cudaMemcpyDeviceToHost, s));
    }
    WL_CUDA_TRY(cudaStreamSynchronize(s));
    if (kind == WL_VEC_XR)
        for (int r = 0; r < n_rhs; ++r) {
            dots[3 * r + 0] = hs[r].rho_re;
            dots[3 * r + 1] = hs[r].rho_im;
            dots[3 * r + 2] = hs[r].rr;
        }
    return checked_result(WL_OK);
}

extern "C" int wl_profile_enable(wl_gauge *g, int on)
{
    if (!g) { set_error("wl_profile_enable: NULL"); return WL_ERR_ARG; }
    std::lock_guard<std::mutex> lock(g->mu);
    g->profiling = on ? 1 : 0;
    std::memset(g->prof, 0, sizeof(g->prof));
    return WL_OK;
}

extern "C" int wl_profile_read(wl_gauge *g, wl_kernel_profile out[4])
{
    if (!g || !out) { set_error("wl_profile_read: NULL"); return WL_ERR_ARG; }
    std::lock_guard<std::mutex> lock(g->mu);
    std::memcpy(out, g->prof, sizeof(g->prof));
    return WL_OK;
}

extern "C" int bicgstab_solve(wl_gauge *g, const void *b, void *x, double m0, const wl_solver_params *p,
                              wl_solver_stats *stats, void *stream)
{
    if (!g || !b || !x || !stats) { set_error("bicgstab_solve: NULL argument"); return WL_ERR_ARG; }
    WL_TRY(check_params(g, p));
    if (!p->eo) { set_error("bicgstab_solve: only the even-odd preconditioned solve is provided"); return WL_ERR_ARG; }
    if (!(2.0 * m0 + 8.0 > 0.0)) { set_error("bicgstab_solve: need 2 m0 + 8 > 0"); return WL_ERR_ARG; }
    std::lock_guard<std::mutex> lock(g->mu);
    cudaStream_t s = as_stream(stream);
    const Geom &geo = g->lat->geom;
    Timer tm;
    const int PO = p->outer_prec;
    Vec be, bo, xe, bprec;
    WL_TRY(make_vec(g, "b_e", PO, 1, &be));
    WL_TRY(make_vec(g, "b_o", PO, 1, &bo));
    WL_TRY(make_vec(g, "x_e", PO, 1, &xe));
    WL_TRY(make_vec(g, "mm_bprec", PO, 1, &bprec));
    const void *bc[1] = {b};
    const void *xc[1] = {x};
    WL_TRY(import_full(geo, bc, be, bo, s));
    WL_TRY(import_spinors(geo, xc, xe, WL_EVEN, s));
    Scratch sc;
    WL_TRY(get_scratch(g, 1, &sc, s));
    std::vector<double> ne, no;
    WL_TRY(norms2_host(g, be, sc, ne, s));
    WL_TRY(norms2_host(g, bo, sc, no, s));
    std::vector<double> bn2 = {ne[0] + no[0]};
    std::vector<wl_solver_stats> st(1);
    std::memset(st.data(), 0, sizeof(wl_solver_stats));
    void *xo[1] = {x};
    WL_TRY(hop(g, bo, bprec, &be, 1.0 / (2.0 * m0 + 8.0), WL_EVEN, 0, 1, s));  // b_e + kappa D_eo b_o
    WL_TRY(solve_one_mass(g, be, bo, bprec, xe, m0, *p, bn2, xo, 1, st, s));
    WL_CUDA_TRY(cudaStreamSynchronize(s));
    st[0].seconds = tm.sec();
    *stats = st[0];
    return checked_result(st[0].status);
}

// Solution-space minimisation guess (Section 6.2.2) for mass m from the
// solutions x_j, j = j0 .. j0+kk-1 in solve order: minimise ||b - M_p(m) psi||
// over psi = sum_j c_j psi_j, psi_j = x_j / (m_j + 4).  With
// M_p(m) psi_j = b + (m - m_j) psi_j = d_j, the normal equations
// sum_j <d_i, d_j> c_j = <d_i, b> need only ||b||^2, <b, x_j> and the Gram
// matrix <x_i, x_j>: with f_i = (m - m_i) / (m_i + 4),
//   <d_i, d_j> = ||b||^2 + f_j <b, x_j> + f_i conj<b, x_i> + f_i f_j <x_i, x_j>,
//   <d_i, b>   = ||b||^2 + f_i conj<b, x_i>.
// Returns the kappa-form weights g_j = c_j (m + 4) / (m_j + 4) of the x_j.
// Solved by Gaussian elimination with partial pivoting in long double; a
// singular system gives the zero guess.
static void ssm_guess(const std::vector<std::vector<std::complex<double>>> &gram,
                      const std::vector<std::complex<double>> &bx, double bn2, double m, const double *m0,
                      const std::vector<int> &order, int j0, int kk, std::vector<std::complex<double>> &g_out)
{
    using C = std::complex<long double>;
    std::vector<std::vector<C>> A(kk, std::vector<C>(kk + 1));
    std::vector<long double> f(kk);
    for (int i = 0; i < kk; ++i) {
        const double mi = m0[order[j0 + i]];
        f[i] = (long double)(m - mi) / (long double)(mi + 4.0);
    }
    for (int i = 0; i < kk; ++i) {
        const C bxi = C(bx[j0 + i]);
        for (int j = 0; j < kk; ++j)
            A[i][j] = (long double)bn2 + f[j] * C(bx[j0 + j]) + f[i] * std::conj(bxi) +
                      f[i] * f[j] * C(gram[j0 + i][j0 + j]);
        A[i][kk] = (long double)bn2 + f[i] * std::conj(bxi);
    }
    for (int c = 0; c < kk; ++c) {
        int piv = c;
        for (int r = c + 1; r < kk; ++r)
            if (std::abs(A[r][c]) > std::abs(A[piv][c])) piv = r;
        if (!(std::abs(A[piv][c]) > 0.0L)) {
            for (auto &v : g_out) v = 0.0;
            return;
        }
        std::swap(A[c], A[piv]);
        for (int r = c + 1; r < kk; ++r) {
            const C fct = A[r][c] / A[c][c];
            for (int q = c; q <= kk; ++q) A[r][q] -= fct * A[c][q];
        }
    }
    std::vector<C> c(kk);
    for (int i = kk - 1; i >= 0; --i) {
        C acc = A[i][kk];
        for (int j = i + 1; j < kk; ++j) acc -= A[i][j] * c[j];
        c[i] = acc / A[i][i];
    }
    for (int j = 0; j < kk; ++j) {
        const double mj = m0[order[j0 + j]];
        const C gj = c[j] * (long double)((m + 4.0) / (mj + 4.0));
        g_out[j] = std::complex<double>((double)gj.real(), (double)gj.imag());
    }
}

extern "C" int multimass_solve(wl_gauge *g, const void *const *b, void *const *x, int n_rhs, const double *m0,
                               int n_mass, const wl_solver_params *p, wl_solver_stats *stats, void *stream)
{
    if (!g || !b || !x || !m0 || !stats || n_rhs < 1 || n_mass < 1 || n_mass > 16) {
        set_error("multimass_solve: bad argument (1 <= n_mass <= 16)");
        return WL_ERR_ARG;
    }
    WL_TRY(check_params(g, p));
    for (int i = 0; i < n_mass; ++i) {
        if (!(2.0 * m0[i] + 8.0 > 0.0)) { set_error("multimass_solve: need 2 m0 + 8 > 0"); return WL_ERR_ARG; }
        for (int j = 0; j < i; ++j)
            if (m0[i] == m0[j]) { set_error("multimass_solve: masses must be distinct"); return WL_ERR_ARG; }
    }
    for (int r = 0; r < n_rhs; ++r)
        if (!b[r]) { set_error("multimass_solve: NULL source"); return WL_ERR_ARG; }
    for (int k = 0; k < n_rhs * n_mass; ++k)
        if (!x[k]) { set_error("multimass_solve: NULL solution pointer"); return WL_ERR_ARG; }
    std::lock_guard<std::mutex> lock(g->mu);
    cudaStream_t s = as_stream(stream);
    const Geom &geo = g->lat->geom;
    const int PO = p->outer_prec;
    Vec be, bo, dbo, bprec;
    WL_TRY(make_vec(g, "b_e", PO, n_rhs, &be));
    WL_TRY(make_vec(g, "b_o", PO, n_rhs, &bo));
    WL_TRY(make_vec(g, "mm_Dbo", PO, n_rhs, &dbo));
    WL_TRY(make_vec(g, "mm_bprec", PO, n_rhs, &bprec));
    WL_TRY(import_full(geo, b, be, bo, s));
    Scratch sc;
    WL_TRY(get_scratch(g, n_rhs, &sc, s));
    std::vector<double> ne, no, bn2(n_rhs);
    WL_TRY(norms2_host(g, be, sc, ne, s));
    WL_TRY(norms2_host(g, bo, sc, no, s));
    for (int r = 0; r < n_rhs; ++r) bn2[r] = ne[r] + no[r];
    // D_eo b_o once for all masses; b_prec(m) = b_e + kappa(m) D_eo b_o.  A
    // source without an odd part (a point source on an even site) needs no
    // hop: its D_eo b_o is zero.  ||b_o||^2 is exactly zero only if every odd
    // entry is below 2.2e-162, whose hop would be as negligible.
    {
        void *pp = nullptr;
        WL_TRY(g->pinned.get("mm_skip", sizeof(int) * n_rhs, &pp));
        int *h_zero = static_cast<int *>(pp);
        int n_zero = 0;
        for (int r = 0; r < n_rhs; ++r) {
            h_zero[r] = no[r] == 0.0 ? 1 : 0;
            n_zero += h_zero[r];
            if (h_zero[r]) WL_CUDA_TRY(cudaMemsetAsync(dbo.rhs(r), 0, dbo.rhs_bytes, s));
        }
        if (n_zero < n_rhs) {
            void *dp = nullptr;
            WL_TRY(g->ws.get("mm_skip", sizeof(int) * n_rhs, &dp));
            WL_CUDA_TRY(cudaMemcpyAsync(dp, h_zero, sizeof(int) * n_rhs, cudaMemcpyHostToDevice, s));
            WL_TRY(hop_ex(g, bo, dbo, nullptr, 0.0, nullptr, 0.0, 1.0, WL_EVEN, 0, 1, static_cast<const int *>(dp), 1,
                          s));
        }
    }

    // heaviest first (Section 7)
    std::vector<int> order(n_mass);
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int a, int c) { return m0[a] > m0[c]; });
    std::vector<Vec> sol(n_mass);  // even-site solutions (outer precision) in solve order
    std::vector<Vec> ys(n_mass);   // y_j = D_eo D_oe x_j of those solutions
    const int ring = (p->guess != WL_GUESS_ZERO && p->guess_max > 0) ? std::min(n_mass, p->guess_max + 1)
                     : p->guess == WL_GUESS_ZERO ? 1 : n_mass;
    std::vector<wl_solver_stats> st(n_rhs);
    void *pin = nullptr;
    WL_TRY(g->pinned.get("mm_coef", sizeof(double) * 128 * n_rhs, &pin));
    double *hc = static_cast<double *>(pin);
    // solution-space minimisation: Gram matrix <x_i, x_j> and <b, x_j> per rhs
    std::vector<std::vector<std::vector<std::complex<double>>>> gram;
    std::vector<std::vector<std::complex<double>>> bx;
    double *ssm_dots = nullptr, *ssm_partials = nullptr;
    unsigned *ssm_tickets = nullptr;
    if (p->guess == WL_GUESS_SSM) {
        gram.assign(n_rhs, std::vector<std::vector<std::complex<double>>>(n_mass,
                                                                          std::vector<std::complex<double>>(n_mass)));
        bx.assign(n_rhs, std::vector<std::complex<double>>(n_mass));
        void *pp;
        const bool fresh = g->ws.bufs["ssm_tickets"].bytes < sizeof(unsigned) * n_rhs;
        WL_TRY(g->ws.get("ssm_tickets", sizeof(unsigned) * n_rhs, &pp));
        ssm_tickets = static_cast<unsigned *>(pp);
        if (fresh) WL_CUDA_TRY(cudaMemsetAsync(pp, 0, sizeof(unsigned) * n_rhs, s));
        WL_TRY(g->ws.get("ssm_partials", sizeof(double) * (2 * 16 * 1024 + 64), &pp));
        ssm_partials = static_cast<double *>(pp);
        WL_TRY(g->ws.get("ssm_dots", sizeof(double) * 2 * 16 * n_rhs, &pp));
        ssm_dots = static_cast<double *>(pp);
    }
    // overlapped exports, except next to the persistent solver's cooperative
    // launch (all its blocks must be resident; nothing else shares the GPU)
    AsyncExport ax;
    AsyncExport *axp = p->mode == WL_MODE_PERSISTENT ? nullptr : &ax;
    if (axp) {
        WL_TRY(ax.init());
        bool host = true;
        for (size_t k = 0; k < (size_t)n_rhs * n_mass && host; ++k) {
            cudaPointerAttributes pa{};
            host = cudaPointerGetAttributes(&pa, x[k]) == cudaSuccess && pa.type == cudaMemoryTypeHost;
        }
        cudaGetLastError();
        // (double-float solutions are converted to FP64 on the way out, which
        // loads the FP64 pipe: their export keeps the full grid)
        if (host && PO == WL_F64) ax.blocks = std::max(1, (ax.blocks + 9) / 10);
    }
    int worst = WL_OK;
    for (int k = 0; k < n_mass; ++k) {
        Timer tm;
        const int im = order[k];
        const double m = m0[im];
        // a guess through the last guess_max masses needs only that many
        // stored solutions: the buffers form a ring of guess_max + 1
        const int slot = k % ring;
        WL_TRY(make_vec(g, "mm_sol" + std::to_string(slot), PO, n_rhs, &sol[k]));
        WL_TRY(make_vec(g, "mm_y" + std::to_string(slot), PO, n_rhs, &ys[k]));
        WL_TRY(blas_xpay(geo, be, 1.0 / (2.0 * m + 8.0), dbo, bprec, s));
        Vec r0;
        WL_TRY(make_vec(g, "dc_r64", PO, n_rhs, &r0));
        const double k2 = 1.0 / ((2.0 * m + 8.0) * (2.0 * m + 8.0));
        // the guess uses the kk most recently solved masses j0 .. k-1 (all
        // of them unless guess_max limits it)
        int kk = (p->guess == WL_GUESS_ZERO) ? 0 : k;
        if (p->guess_max > 0) kk = std::min(kk, p->guess_max);
        const int j0 = k - kk;
        const bool ssm = p->guess == WL_GUESS_SSM && kk > 0;
        // x_guess = sum_j g_j x_j (g_j real for POLY, complex for SSM); by
        // linearity the first residual b_prec - x_guess + kappa^2 sum_j g_j y_j,
        // with y_j = D_eo D_oe x_j kept from mass j, needs no hop.
        // Coefficients: g_j at coef[r kk + j], kappa^2 g_j at coef[32 n_rhs + r kk + j]
        // (complex: re, im pairs).
        if (!ssm) {
            // Lagrange extrapolation of psi = x / (m + 4) (Eq. Poly):
            // g_j = (m + 4) w_j / (m_j + 4), w_j = prod_{i != j} (m - m_i) / (m_j - m_i)
            std::vector<double> cj(kk);
            for (int j = 0; j < kk; ++j) {
                const double mj = m0[order[j0 + j]];
                double w = 1.0;
                for (int i = 0; i < kk; ++i)
                    if (i != j) {
                        const double mi = m0[order[j0 + i]];
                        w *= (m - mi) / (mj - mi);
                    }
                cj[j] = (m + 4.0) * w / (mj + 4.0);
            }
            for (int r = 0; r < n_rhs; ++r)
                for (int j = 0; j < kk; ++j) {
                    hc[r * kk + j] = cj[j];
                    hc[32 * n_rhs + r * kk + j] = k2 * cj[j];
                }
        } else {
            for (int r = 0; r < n_rhs; ++r) {
                std::vector<std::complex<double>> gj(kk);
                ssm_guess(gram[r], bx[r], bn2[r], m, m0, order, j0, kk, gj);
                for (int j = 0; j < kk; ++j) {
                    const std::complex<double> d = k2 * gj[j];
                    hc[2 * (r * kk + j)] = gj[j].real();
                    hc[2 * (r * kk + j) + 1] = gj[j].imag();
                    hc[32 * n_rhs + 2 * (r * kk + j)] = d.real();
                    hc[32 * n_rhs + 2 * (r * kk + j) + 1] = d.imag();
                }
            }
        }
        if (kk > 0) WL_CUDA_TRY(cudaMemcpyAsync(sc.coef, hc, sizeof(double) * 64 * n_rhs, cudaMemcpyHostToDevice, s));
        {
            // x_guess and the first residual in one pass over the stored x_j, y_j
            std::vector<const Vec *> ins(2 * kk + 1);
            for (int j = 0; j < kk; ++j) {
                ins[j] = &sol[j0 + j];
                ins[kk + j] = &ys[j0 + j];
            }
            ins[2 * kk] = &bprec;
            WL_TRY(blas_guess_residual(geo, sc.coef, sc.coef + 32 * n_rhs, ins.data(), kk, sol[k], r0, s, ssm));
        }
        for (int r = 0; r < n_rhs; ++r) std::memset(&st[r], 0, sizeof(wl_solver_stats));
        // nothing overlaps the last mass's export: give it the whole GPU
        if (axp && k == n_mass - 1) ax.blocks = ax.full_blocks;
        WL_TRY(solve_one_mass(g, be, bo, bprec, sol[k], m, *p, bn2, x + im, n_mass, st, s, &ys[k], true, axp));
        if (p->guess == WL_GUESS_SSM && k + 1 < n_mass) {
            // the Gram products read the canonical solutions: wait for their export
            WL_TRY(ax.join(s));
            // Gram data of the new solution x_k for later masses:
            // <b, x_k> and <x_j, x_k>, j <= k, on the canonical outputs
            const int n = k + 2;
            std::vector<const void *> a(n_rhs), in((size_t)n_rhs * n);
            for (int r = 0; r < n_rhs; ++r) {
                a[r] = x[(size_t)r * n_mass + im];
                in[(size_t)r * n] = b[r];
                for (int j = 0; j <= k; ++j) in[(size_t)r * n + 1 + j] = x[(size_t)r * n_mass + order[j]];
            }
            WL_TRY(canon_dots(a.data(), in.data(), n, n_rhs, (size_t)geo.Vh * 2 * 12, ssm_dots, ssm_partials,
                              ssm_tickets, s));
            std::vector<double> hd(2 * (size_t)n * n_rhs);
            WL_CUDA_TRY(cudaMemcpyAsync(hd.data(), ssm_dots, sizeof(double) * hd.size(), cudaMemcpyDeviceToHost, s));
            WL_CUDA_TRY(cudaStreamSynchronize(s));
            for (int r = 0; r < n_rhs; ++r) {
                const double *d = hd.data() + 2 * (size_t)n * r;
                bx[r][k] = {d[0], d[1]};
                for (int j = 0; j <= k; ++j) {
                    gram[r][j][k] = {d[2 + 2 * j], d[3 + 2 * j]};
                    gram[r][k][j] = std::conj(gram[r][j][k]);
                }
            }
        }
        WL_CUDA_TRY(cudaStreamSynchronize(s));
        const double sec = tm.sec();
        for (int r = 0; r < n_rhs; ++r) {
            st[r].seconds = sec;
            stats[(size_t)r * n_mass + im] = st[r];
            if (st[r].status != WL_OK) worst = st[r].status;
        }
    }
    WL_TRY(ax.join(s));
    WL_CUDA_TRY(cudaStreamSynchronize(s));
    return checked_result(worst);
}
