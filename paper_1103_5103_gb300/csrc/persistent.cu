// Persistent fused BiCGstab (WL_MODE_PERSISTENT): one cooperative launch runs
// whole iterations of the inner solve for every right-hand side.  The seven
// steps of an iteration (see solver.cu) become phases of one kernel,
// separated by a grid barrier; the reductions are accumulated per block in
// shared memory, added to per-rhs FP64 totals with atomics, and the block
// that arrives last at the barrier evaluates the scalar recurrences before
// releasing the others -- so no phase needs a second barrier and no step
// returns to the host.
//
// Every barrier wait is bounded: a block that spins past the deadline sets
// an error word and returns, and the blocks still waiting then time out in
// turn, so a lost arrival ends the kernel with WL_ERR_TIMEOUT instead of
// hanging the GPU.  The launch is cooperative, which guarantees that all
// blocks are resident together.
//
// Totals are summed with FP64 atomics, so their rounding order -- and hence
// the last bits of the iterates -- can differ from run to run; the graph
// mode is the bit-reproducible one.
#include <cstring>
#include <string>

#include "hop.cuh"

namespace wl {

constexpr int kPersistMaxRhs = 32;

struct PersistCtl {
    unsigned count;     // arrivals at the current barrier
    unsigned gen;       // barrier generation
    int err;            // 1: a barrier wait timed out
    int skip_arrival;   // test hook: block 0 skips its first arrival (the others then time out)
    long long deadline; // spin limit in SM clock cycles
    double acc[kPersistMaxRhs][4];  // per-rhs reduction totals
};

struct PersistArgs {
    HopArgs hop_odd;    // D_oe: in = p or s (set per phase), out parity odd
    HopArgs hop_even;   // D_eo on tmp
    Vec r, rhat, p, v, s, t, tmp, e;
    BiState *st;
    const double *kappa2;  // -kappa^2
    PersistCtl *ctl;
    int nrhs, max_iter;
};

__device__ __forceinline__ int ld_volatile(const int *p) { return *(volatile const int *)p; }

// State written by one block and read by others between barriers (BiState,
// the totals, the barrier words) is accessed through volatile lvalues, and
// every vector the kernel rewrites is read with ordinary loads (ordered by
// the barrier's fences), never through the non-coherent read-only path.

// Grid barrier with a bounded spin.  fin(), if given, runs in thread 0 of
// the last block to arrive, before the others are released.  Returns false
// when any block has timed out.
template <class Fin>
__device__ __forceinline__ bool grid_barrier(PersistCtl *c, Fin fin)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        const unsigned g0 = *(volatile unsigned *)&c->gen;
        __threadfence();
        const bool skip = c->skip_arrival && blockIdx.x == 0;
        if (skip) c->skip_arrival = 0;
        const unsigned arrived = skip ? 0u : atomicAdd(&c->count, 1u);
        if (!skip && arrived == gridDim.x - 1) {
            fin();
            c->count = 0;
            __threadfence();
            atomicAdd(&c->gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*(volatile unsigned *)&c->gen == g0) {
                if (ld_volatile(&c->err) || clock64() - t0 > c->deadline) {
                    atomicExch(&c->err, 1);
                    break;
                }
            }
        }
        __threadfence();
        if (ld_volatile(&c->err)) ok = 0;
    }
    __syncthreads();
    return ok != 0;
}

struct NoFin {
    __device__ void operator()() const {}
};

// Per-block, per-rhs accumulation of NV values (thread 0 holds the block sums).
template <int NV>
__device__ __forceinline__ void block_add(double (&v)[NV], double (*sacc)[4], int r)
{
    block_sum<NV>(v);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sacc[r][k] += v[k];
}

__device__ __forceinline__ void flush_acc(double (*sacc)[4], PersistCtl *c, int nrhs, int nv)
{
    if (threadIdx.x == 0)
        for (int r = 0; r < nrhs; ++r)
            for (int k = 0; k < nv; ++k) {
                if (sacc[r][k] != 0.0) atomicAdd(&c->acc[r][k], sacc[r][k]);
                sacc[r][k] = 0.0;
            }
}

constexpr int kPersistBlock = 384;  // one block per SM: fewer arrivals per barrier

template <int P, int PX>
__global__ void __launch_bounds__(kPersistBlock, 1) k_bicgstab_persistent(PersistArgs A)
{
    using R = typename PrecTraits<P>::R;
    using RX = typename PrecTraits<PX>::R;
    __shared__ double sacc[kPersistMaxRhs][4];
    for (int k = threadIdx.x; k < kPersistMaxRhs * 4; k += blockDim.x) (&sacc[0][0])[k] = 0.0;
    __syncthreads();
    const Geom &g = A.hop_odd.g;
    const int nsb = (g.Vh + kPersistBlock - 1) / kPersistBlock;
    const int nunits = nsb * A.nrhs;
    PersistCtl *c = A.ctl;
    BiState *st = A.st;
    auto done = [&](int r) { return ld_volatile(&st[r].done) != 0; };
    auto unit = [&](int u, int &r, int &i) {
        r = u % A.nrhs;
        i = (u / A.nrhs) * kPersistBlock + threadIdx.x;
    };
    for (int it = 0; it < A.max_iter; ++it) {
        bool all = true;
        for (int r = 0; r < A.nrhs; ++r) all &= done(r);
        if (all) break;
        const double k2 = *(volatile const double *)A.kappa2;
        // 1: tmp = D_oe p
        for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
            int r, i;
            unit(u, r, i);
            if (done(r) || i >= g.Vh) continue;
            HopArgs h = A.hop_odd;
            h.in = A.p.ptr;
            cx<R> acc[1][12];
#pragma unroll
            for (int k = 0; k < 12; ++k) acc[0][k] = acc_zero<R>();
            hop_accumulate<P, false, 1, true>(h, i, r, acc);
            SpinorIO<P>::store(A.tmp.rhs(r), g.stride, i, acc[0]);
        }
        if (!grid_barrier(c, NoFin{})) return;
        // 2: v = p - k^2 D_eo tmp, <rhat, v> -> alpha
        for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
            int r, i;
            unit(u, r, i);
            if (done(r)) continue;
            double red[2] = {0.0, 0.0};
            if (i < g.Vh) {
                cx<R> acc[1][12];
#pragma unroll
                for (int k = 0; k < 12; ++k) acc[0][k] = acc_zero<R>();
                hop_accumulate<P, false, 1, true>(A.hop_even, i, r, acc);
                cx<R> pv[12], o[12], rh[12];
                SpinorIO<P>::template load<true>(A.p.rhs(r), g.stride, i, pv);
#pragma unroll
                for (int k = 0; k < 12; ++k) o[k] = pv[k] + R(k2) * acc[0][k];
                SpinorIO<P>::roundtrip(o);
                SpinorIO<P>::store(A.v.rhs(r), g.stride, i, o);
                SpinorIO<P>::template load<true>(A.rhat.rhs(r), g.stride, i, rh);
                cx<R> d = {R(0), R(0)};
#pragma unroll
                for (int k = 0; k < 12; ++k) d = conjmad(rh[k], o[k], d);
                red[0] = d.re;
                red[1] = d.im;
            }
            block_add<2>(red, sacc, r);
        }
        flush_acc(sacc, c, A.nrhs, 2);
        if (!grid_barrier(c, [&] {
                volatile double(*acc)[4] = c->acc;
                for (int r = 0; r < A.nrhs; ++r) {
                    volatile BiState &S = st[r];
                    const double dr = acc[r][0], di = acc[r][1];
                    acc[r][0] = acc[r][1] = 0.0;
                    if (S.done) continue;
                    const double den = dr * dr + di * di;
                    if (!(den > 0.0) || !isfinite(den)) {
                        S.breakdown = 1;
                        S.done = 1;
                    } else {
                        S.alpha_re = (S.rho_re * dr + S.rho_im * di) / den;
                        S.alpha_im = (S.rho_im * dr - S.rho_re * di) / den;
                    }
                }
            }))
            return;
        // 3: s = r - alpha v
        for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
            int r, i;
            unit(u, r, i);
            if (done(r) || i >= g.Vh) continue;
            const cx<R> al = {R(*(volatile double *)&st[r].alpha_re), R(*(volatile double *)&st[r].alpha_im)};
            cx<R> a[12], b[12];
            SpinorIO<P>::template load<true>(A.r.rhs(r), g.stride, i, a);
            SpinorIO<P>::template load<true>(A.v.rhs(r), g.stride, i, b);
#pragma unroll
            for (int k = 0; k < 12; ++k) a[k] = a[k] - al * b[k];
            SpinorIO<P>::store(A.s.rhs(r), g.stride, i, a);
        }
        if (!grid_barrier(c, NoFin{})) return;
        // 4: tmp = D_oe s
        for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
            int r, i;
            unit(u, r, i);
            if (done(r) || i >= g.Vh) continue;
            HopArgs h = A.hop_odd;
            h.in = A.s.ptr;
            cx<R> acc[1][12];
#pragma unroll
            for (int k = 0; k < 12; ++k) acc[0][k] = acc_zero<R>();
            hop_accumulate<P, false, 1, true>(h, i, r, acc);
            SpinorIO<P>::store(A.tmp.rhs(r), g.stride, i, acc[0]);
        }
        if (!grid_barrier(c, NoFin{})) return;
        // 5: t = s - k^2 D_eo tmp, <t, s>, <t, t> -> omega
        for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
            int r, i;
            unit(u, r, i);
            if (done(r)) continue;
            double red[3] = {0.0, 0.0, 0.0};
            if (i < g.Vh) {
                cx<R> acc[1][12];
#pragma unroll
                for (int k = 0; k < 12; ++k) acc[0][k] = acc_zero<R>();
                hop_accumulate<P, false, 1, true>(A.hop_even, i, r, acc);
                cx<R> sv[12], o[12];
                SpinorIO<P>::template load<true>(A.s.rhs(r), g.stride, i, sv);
#pragma unroll
                for (int k = 0; k < 12; ++k) o[k] = sv[k] + R(k2) * acc[0][k];
                SpinorIO<P>::roundtrip(o);
                SpinorIO<P>::store(A.t.rhs(r), g.stride, i, o);
                cx<R> d = {R(0), R(0)};
                R n = R(0);
#pragma unroll
                for (int k = 0; k < 12; ++k) {
                    d = conjmad(o[k], sv[k], d);
                    n = fma(o[k].re, o[k].re, fma(o[k].im, o[k].im, n));
                }
                red[0] = d.re;
                red[1] = d.im;
                red[2] = n;
            }
            block_add<3>(red, sacc, r);
        }
        flush_acc(sacc, c, A.nrhs, 3);
        if (!grid_barrier(c, [&] {
                volatile double(*acc)[4] = c->acc;
                for (int r = 0; r < A.nrhs; ++r) {
                    volatile BiState &S = st[r];
                    const double a = acc[r][0], b = acc[r][1], tt = acc[r][2];
                    acc[r][0] = acc[r][1] = acc[r][2] = 0.0;
                    if (S.done) continue;
                    if (tt > 0.0 && isfinite(tt)) {
                        S.omega_re = a / tt;
                        S.omega_im = b / tt;
                    } else {
                        S.omega_re = S.omega_im = 0.0;
                    }
                }
            }))
            return;
        // 6: x += alpha p + omega s; r = s - omega t; <rhat, r>, ||r||^2 -> beta
        for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
            int r, i;
            unit(u, r, i);
            if (done(r)) continue;
            double red[3] = {0.0, 0.0, 0.0};
            if (i < g.Vh) {
                const BiState &S = st[r];
                const double are = *(volatile const double *)&S.alpha_re, aim = *(volatile const double *)&S.alpha_im;
                const double ore = *(volatile const double *)&S.omega_re, oim = *(volatile const double *)&S.omega_im;
                cx<R> pv[12], sv[12], tv[12];
                SpinorIO<P>::template load<true>(A.p.rhs(r), g.stride, i, pv);
                SpinorIO<P>::template load<true>(A.s.rhs(r), g.stride, i, sv);
                SpinorIO<P>::template load<true>(A.t.rhs(r), g.stride, i, tv);
                cx<RX> xv[12];
                SpinorIO<PX>::template load<true>(A.e.rhs(r), g.stride, i, xv);
                const cx<RX> al = {(RX)are, (RX)aim}, om = {(RX)ore, (RX)oim};
#pragma unroll
                for (int k = 0; k < 12; ++k) {
                    const cx<RX> pk = {(RX)pv[k].re, (RX)pv[k].im}, sk = {(RX)sv[k].re, (RX)sv[k].im};
                    xv[k] = cmad(al, pk, cmad(om, sk, xv[k]));
                }
                SpinorIO<PX>::store(A.e.rhs(r), g.stride, i, xv);
                const cx<R> omr = {(R)ore, (R)oim};
                cx<R> rv[12], rh[12];
#pragma unroll
                for (int k = 0; k < 12; ++k) rv[k] = sv[k] - omr * tv[k];
                SpinorIO<P>::roundtrip(rv);
                SpinorIO<P>::store(A.r.rhs(r), g.stride, i, rv);
                SpinorIO<P>::template load<true>(A.rhat.rhs(r), g.stride, i, rh);
                cx<R> d = {R(0), R(0)};
                R n = R(0);
#pragma unroll
                for (int k = 0; k < 12; ++k) {
                    d = conjmad(rh[k], rv[k], d);
                    n = fma(rv[k].re, rv[k].re, fma(rv[k].im, rv[k].im, n));
                }
                red[0] = d.re;
                red[1] = d.im;
                red[2] = n;
            }
            block_add<3>(red, sacc, r);
        }
        flush_acc(sacc, c, A.nrhs, 3);
        if (!grid_barrier(c, [&] {
                volatile double(*acc)[4] = c->acc;
                for (int r = 0; r < A.nrhs; ++r) {
                    volatile BiState &S = st[r];
                    const double r1re = acc[r][0], r1im = acc[r][1], rr = acc[r][2];
                    acc[r][0] = acc[r][1] = acc[r][2] = 0.0;
                    if (S.done) continue;
                    S.iters += 1;
                    S.rr = rr;
                    const double ore = S.omega_re, oim = S.omega_im;
                    if (!isfinite(rr) || !isfinite(r1re) || !isfinite(r1im)) {
                        S.breakdown = 1;
                        S.done = 1;
                    } else if (rr <= S.target2) {
                        S.done = 1;
                    } else {
                        const double rho2 = S.rho_re * S.rho_re + S.rho_im * S.rho_im;
                        const double om2 = ore * ore + oim * oim;
                        if (!(rho2 > 0.0) || !(om2 > 0.0) || !(r1re * r1re + r1im * r1im > 0.0)) {
                            S.breakdown = 1;
                            S.done = 1;
                        } else {
                            const double qre = (r1re * S.rho_re + r1im * S.rho_im) / rho2;
                            const double qim = (r1im * S.rho_re - r1re * S.rho_im) / rho2;
                            const double are = S.alpha_re, aim = S.alpha_im;
                            const double wre = (are * ore + aim * oim) / om2;
                            const double wim = (aim * ore - are * oim) / om2;
                            S.beta_re = qre * wre - qim * wim;
                            S.beta_im = qre * wim + qim * wre;
                            S.rho_re = r1re;
                            S.rho_im = r1im;
                        }
                    }
                }
            }))
            return;
        // 7: p = r + beta (p - omega v)
        for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
            int r, i;
            unit(u, r, i);
            if (done(r) || i >= g.Vh) continue;
            const BiState &S = st[r];
            const cx<R> be = {(R)*(volatile const double *)&S.beta_re, (R)*(volatile const double *)&S.beta_im};
            const cx<R> om = {(R)*(volatile const double *)&S.omega_re, (R)*(volatile const double *)&S.omega_im};
            cx<R> rv[12], pv[12], vv[12];
            SpinorIO<P>::template load<true>(A.r.rhs(r), g.stride, i, rv);
            SpinorIO<P>::template load<true>(A.p.rhs(r), g.stride, i, pv);
            SpinorIO<P>::template load<true>(A.v.rhs(r), g.stride, i, vv);
#pragma unroll
            for (int k = 0; k < 12; ++k) pv[k] = rv[k] + be * (pv[k] - om * vv[k]);
            SpinorIO<P>::store(A.p.rhs(r), g.stride, i, pv);
        }
        if (!grid_barrier(c, NoFin{})) return;
    }
}

template <int P, int PX>
static int launch_persistent_t(PersistArgs &A, cudaStream_t s)
{
    int dev = 0, nsm = 0, per = 0;
    WL_CUDA_TRY(cudaGetDevice(&dev));
    WL_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    WL_CUDA_TRY(
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_bicgstab_persistent<P, PX>, kPersistBlock, 0));
    if (per < 1) { set_error("persistent solver: kernel cannot be resident"); return WL_ERR_CUDA; }
    const int nsb = (A.hop_odd.g.Vh + kPersistBlock - 1) / kPersistBlock;
    int grid = nsm * per;
    if (grid > nsb * A.nrhs) grid = nsb * A.nrhs;
    void *args[] = {&A};
    WL_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)k_bicgstab_persistent<P, PX>, dim3(grid),
                                            dim3(kPersistBlock), args, 0, s));
    note_launch(s);
    return WL_OK;
}

// Run up to max_iter inner iterations in one cooperative launch.  Returns
// WL_ERR_TIMEOUT if a barrier wait ran out (the kernel then exits; the
// solver state is left as it was at that barrier).
int persistent_inner(wl_gauge *g, int prec, int nrhs, const Vec &r, const Vec &rhat, const Vec &p, const Vec &v,
                     const Vec &sv, const Vec &t, const Vec &tmp, const Vec &e, BiState *state, const double *kappa2,
                     int max_iter, double deadline_s, int skip_arrival, cudaStream_t s)
{
    if (nrhs > kPersistMaxRhs) {
        set_error("persistent solver: at most 32 right-hand sides");
        return WL_ERR_ARG;
    }
    void *pc;
    WL_TRY(g->ws.get("persist_ctl", sizeof(PersistCtl), &pc));
    PersistCtl *ctl = static_cast<PersistCtl *>(pc);
    int dev = 0, khz = 0;
    WL_CUDA_TRY(cudaGetDevice(&dev));
    WL_CUDA_TRY(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev));
    PersistCtl h;
    std::memset(&h, 0, sizeof(h));
    h.deadline = (long long)(deadline_s * (khz > 0 ? khz : 2000000) * 1e3);
    h.skip_arrival = skip_arrival;
    WL_CUDA_TRY(cudaMemcpyAsync(ctl, &h, sizeof(h), cudaMemcpyHostToDevice, s));
    PersistArgs A;
    const Geom &geo = g->lat->geom;
    HopArgs &ho = A.hop_odd;
    ho.g = geo;
    ho.out_parity = WL_ODD;
    ho.nrhs = ho.ngroups = nrhs;
    ho.in = p.ptr;
    ho.rhs_bytes = p.rhs_bytes;
    ho.links_out = g->links[prec_index(prec)][WL_ODD];
    ho.links_in = g->links[prec_index(prec)][WL_EVEN];
    ho.skip = nullptr;
    ho.skip_stride = 0;
    HopArgs &he = A.hop_even;
    he = ho;
    he.out_parity = WL_EVEN;
    he.in = tmp.ptr;
    he.links_out = g->links[prec_index(prec)][WL_EVEN];
    he.links_in = g->links[prec_index(prec)][WL_ODD];
    A.r = r; A.rhat = rhat; A.p = p; A.v = v; A.s = sv; A.t = t; A.tmp = tmp; A.e = e;
    A.st = state;
    A.kappa2 = kappa2;
    A.ctl = ctl;
    A.nrhs = nrhs;
    A.max_iter = max_iter;
    if (prec == WL_F32) { WL_TRY((launch_persistent_t<WL_F32, WL_F32>(A, s))); }
    else if (prec == WL_F16) { WL_TRY((launch_persistent_t<WL_F16, WL_F32>(A, s))); }
    else if (prec == WL_F64) { WL_TRY((launch_persistent_t<WL_F64, WL_F64>(A, s))); }
    else { set_error("persistent solver: bad precision"); return WL_ERR_ARG; }
    int err = 0;
    WL_CUDA_TRY(cudaMemcpyAsync(&err, &ctl->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    WL_CUDA_TRY(cudaStreamSynchronize(s));
    if (err) {
        set_error("persistent solver: a grid barrier wait ran out");
        return WL_ERR_TIMEOUT;
    }
    return WL_OK;
}

}  // namespace wl
