// Fused vector kernels of the solvers (Section 5): each BiCGstab update is one
// pass over the site-blocked vectors, with its inner products reduced in the
// same pass (per-site FP32/FP64 partials, FP64 across sites and blocks) and
// the scalar recurrences evaluated on the device by the last block.
//
// Grid convention of every kernel here: blockIdx.x = site_block * nrhs + rhs,
// kBlock threads, one site per thread.
#include "internal.h"

namespace wl {

template <int P>
using RT = typename PrecTraits<P>::R;

struct SiteIdx {
    int r, sb, nsb, i;
};

__device__ __forceinline__ SiteIdx site_idx(int nrhs)
{
    SiteIdx s;
    s.r = blockIdx.x % nrhs;
    s.sb = blockIdx.x / nrhs;
    s.nsb = gridDim.x / nrhs;
    s.i = s.sb * blockDim.x + threadIdx.x;
    return s;
}

template <int P>
__device__ __forceinline__ void ld(const Vec &v, int r, int stride, int i, cx<RT<P>> (&o)[12])
{
    SpinorIO<P>::load(v.rhs(r), stride, i, o);
}

template <int P>
__device__ __forceinline__ void st(const Vec &v, int r, int stride, int i, const cx<RT<P>> (&o)[12])
{
    SpinorIO<P>::store(v.rhs(r), stride, i, o);
}

static inline int grid_of(const Geom &g, int nrhs) { return site_blocks(g) * nrhs; }

// ------------------------------------------------------------ s = r - alpha v

template <int P>
__global__ void __launch_bounds__(kBlock) k_s_update(Geom g, Vec r, Vec v, Vec s, const BiState *state)
{
    const SiteIdx q = site_idx(r.nrhs);
    if (__ldcg(&state[q.r].done) || q.i >= g.Vh) return;
    using R = RT<P>;
    const cx<R> al = {(R)__ldcg(&state[q.r].alpha_re), (R)__ldcg(&state[q.r].alpha_im)};
    cx<R> a[12], b[12];
    ld<P>(r, q.r, g.stride, q.i, a);
    ld<P>(v, q.r, g.stride, q.i, b);
#pragma unroll
    for (int k = 0; k < 12; ++k) a[k] = a[k] - al * b[k];
    st<P>(s, q.r, g.stride, q.i, a);
}

int blas_s_update(const Geom &g, const Vec &r, const Vec &v, const Vec &s_out, BiState *state, cudaStream_t s)
{
    switch (r.prec) {
    case WL_F64: k_s_update<WL_F64><<<grid_of(g, r.nrhs), kBlock, 0, s>>>(g, r, v, s_out, state); break;
    case WL_F32: k_s_update<WL_F32><<<grid_of(g, r.nrhs), kBlock, 0, s>>>(g, r, v, s_out, state); break;
    case WL_F16: k_s_update<WL_F16><<<grid_of(g, r.nrhs), kBlock, 0, s>>>(g, r, v, s_out, state); break;
    }
    WL_CUDA_TRY(cudaGetLastError());
    note_launch(s);
    return WL_OK;
}

// ------------------------------- x += alpha p + omega s;  r = s - omega t
// reductions: <rhat, r> and ||r||^2 -> beta, rho, convergence

template <int P, int PX>
__global__ void __launch_bounds__(kBlock) k_xr_update(Geom g, Vec x, Vec p, Vec sv, Vec t, Vec r, Vec rhat,
                                                      BiState *state, double *partials)
{
    const SiteIdx q = site_idx(r.nrhs);
    BiState &S = state[q.r];
    if (__ldcg(&S.done)) return;
    using R = RT<P>;
    using RX = RT<PX>;
    using RedT = typename RedType<R>::T;
    RedT red[3] = {RedT(0), RedT(0), RedT(0)};
    if (q.i < g.Vh) {
        const double are = __ldcg(&S.alpha_re), aim = __ldcg(&S.alpha_im);
        const double ore = __ldcg(&S.omega_re), oim = __ldcg(&S.omega_im);
        cx<R> pv[12], sv_[12], tv[12];
        ld<P>(p, q.r, g.stride, q.i, pv);
        ld<P>(sv, q.r, g.stride, q.i, sv_);
        ld<P>(t, q.r, g.stride, q.i, tv);
        {
            cx<RX> xv[12];
            SpinorIO<PX>::load(x.rhs(q.r), g.stride, q.i, xv);
            const cx<RX> al = {(RX)are, (RX)aim}, om = {(RX)ore, (RX)oim};
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                cx<RX> pk = {(RX)pv[k].re, (RX)pv[k].im}, sk = {(RX)sv_[k].re, (RX)sv_[k].im};
                xv[k] = cmad(al, pk, cmad(om, sk, xv[k]));
            }
            SpinorIO<PX>::store(x.rhs(q.r), g.stride, q.i, xv);
        }
        const cx<R> om = {(R)ore, (R)oim};
        cx<R> rv[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) rv[k] = sv_[k] - om * tv[k];
        SpinorIO<P>::store_rounded(r.rhs(q.r), g.stride, q.i, rv);
        cx<R> rh[12];
        ld<P>(rhat, q.r, g.stride, q.i, rh);
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
    double tot[3];
    if (grid_sum<3>(red, partials + (size_t)q.r * q.nsb * kRedNV, &S.ticket[2], q.sb, q.nsb, tot) &&
        threadIdx.x == 0) {
        const double r1re = tot[0], r1im = tot[1], rr = tot[2];
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
            if (!(rho2 > 0.0) || !(om2 > 0.0) || !(r1re * r1re + r1im * r1im > S.brk2 * S.rhat2 * rr)) {
                S.breakdown = 1;
                S.done = 1;
            } else {
                // beta = (rho1 / rho) * (alpha / omega)
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
}

int blas_xr_update(const Geom &g, const Vec &x, const Vec &p, const Vec &sv, const Vec &t, const Vec &r,
                   const Vec &rhat, BiState *state, double *partials, cudaStream_t s)
{
    const int gr = grid_of(g, r.nrhs);
    if (r.prec == WL_F64 && x.prec == WL_F64)
        k_xr_update<WL_F64, WL_F64><<<gr, kBlock, 0, s>>>(g, x, p, sv, t, r, rhat, state, partials);
    else if (r.prec == WL_F32 && x.prec == WL_F32)
        k_xr_update<WL_F32, WL_F32><<<gr, kBlock, 0, s>>>(g, x, p, sv, t, r, rhat, state, partials);
    else if (r.prec == WL_F16 && x.prec == WL_F32)
        k_xr_update<WL_F16, WL_F32><<<gr, kBlock, 0, s>>>(g, x, p, sv, t, r, rhat, state, partials);
    else {
        set_error("blas_xr_update: unsupported precision pair");
        return WL_ERR_ARG;
    }
    WL_CUDA_TRY(cudaGetLastError());
    note_launch(s);
    return WL_OK;
}

// ------------------- CG on the normal equations: x += alpha p, r -= alpha w
// with ||r||^2 for the stopping test (the true inner residual r = b - M x,
// not the normal-equation residual).

template <int P, int PX>
__global__ void __launch_bounds__(kBlock) k_cg_xr(Geom g, Vec x, Vec p, Vec w, Vec r, BiState *state,
                                                  double *partials)
{
    const SiteIdx q = site_idx(r.nrhs);
    BiState &S = state[q.r];
    if (__ldcg(&S.done)) return;
    using R = RT<P>;
    using RX = RT<PX>;
    using RedT = typename RedType<R>::T;
    RedT red[1] = {RedT(0)};
    if (q.i < g.Vh) {
        const double al = __ldcg(&S.alpha_re);
        cx<R> pv[12], wv[12], rv[12];
        ld<P>(p, q.r, g.stride, q.i, pv);
        ld<P>(w, q.r, g.stride, q.i, wv);
        ld<P>(r, q.r, g.stride, q.i, rv);
        cx<RX> xv[12];
        SpinorIO<PX>::load(x.rhs(q.r), g.stride, q.i, xv);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            xv[k] = {fma((RX)al, (RX)pv[k].re, xv[k].re), fma((RX)al, (RX)pv[k].im, xv[k].im)};
            rv[k] = {fma(-(R)al, wv[k].re, rv[k].re), fma(-(R)al, wv[k].im, rv[k].im)};
        }
        SpinorIO<PX>::store(x.rhs(q.r), g.stride, q.i, xv);
        SpinorIO<P>::store_rounded(r.rhs(q.r), g.stride, q.i, rv);
        R n = R(0);
#pragma unroll
        for (int k = 0; k < 12; ++k) n = fma(rv[k].re, rv[k].re, fma(rv[k].im, rv[k].im, n));
        red[0] = n;
    }
    double tot[1];
    if (grid_sum<1>(red, partials + (size_t)q.r * q.nsb * kRedNV, &S.ticket[1], q.sb, q.nsb, tot) &&
        threadIdx.x == 0) {
        const double rr = tot[0];
        S.iters += 1;
        S.rr = rr;
        if (!isfinite(rr)) {
            S.breakdown = 1;
            S.done = 1;
        } else if (rr <= S.target2) {
            S.done = 1;
        }
    }
}

int blas_cg_xr(const Geom &g, const Vec &x, const Vec &p, const Vec &w, const Vec &r, BiState *state,
               double *partials, cudaStream_t s)
{
    const int gr = grid_of(g, r.nrhs);
    if (r.prec == WL_F64 && x.prec == WL_F64)
        k_cg_xr<WL_F64, WL_F64><<<gr, kBlock, 0, s>>>(g, x, p, w, r, state, partials);
    else if (r.prec == WL_F32 && x.prec == WL_F32)
        k_cg_xr<WL_F32, WL_F32><<<gr, kBlock, 0, s>>>(g, x, p, w, r, state, partials);
    else if (r.prec == WL_F16 && x.prec == WL_F32)
        k_cg_xr<WL_F16, WL_F32><<<gr, kBlock, 0, s>>>(g, x, p, w, r, state, partials);
    else {
        set_error("blas_cg_xr: unsupported precision pair");
        return WL_ERR_ARG;
    }
    WL_CUDA_TRY(cudaGetLastError());
    note_launch(s);
    return WL_OK;
}

// ------------------------------------------------ p = r + beta (p - omega v)

template <int P>
__global__ void __launch_bounds__(kBlock) k_p_update(Geom g, Vec r, Vec p, Vec v, const BiState *state)
{
    const SiteIdx q = site_idx(r.nrhs);
    if (__ldcg(&state[q.r].done) || q.i >= g.Vh) return;
    using R = RT<P>;
    const cx<R> be = {(R)__ldcg(&state[q.r].beta_re), (R)__ldcg(&state[q.r].beta_im)};
    const cx<R> om = {(R)__ldcg(&state[q.r].omega_re), (R)__ldcg(&state[q.r].omega_im)};
    cx<R> rv[12], pv[12], vv[12];
    ld<P>(r, q.r, g.stride, q.i, rv);
    ld<P>(p, q.r, g.stride, q.i, pv);
    ld<P>(v, q.r, g.stride, q.i, vv);
#pragma unroll
    for (int k = 0; k < 12; ++k) pv[k] = rv[k] + be * (pv[k] - om * vv[k]);
    st<P>(p, q.r, g.stride, q.i, pv);
}

int blas_p_update(const Geom &g, const Vec &r, const Vec &p, const Vec &v, BiState *state, cudaStream_t s)
{
    switch (r.prec) {
    case WL_F64: k_p_update<WL_F64><<<grid_of(g, r.nrhs), kBlock, 0, s>>>(g, r, p, v, state); break;
    case WL_F32: k_p_update<WL_F32><<<grid_of(g, r.nrhs), kBlock, 0, s>>>(g, r, p, v, state); break;
    case WL_F16: k_p_update<WL_F16><<<grid_of(g, r.nrhs), kBlock, 0, s>>>(g, r, p, v, state); break;
    }
    WL_CUDA_TRY(cudaGetLastError());
    note_launch(s);
    return WL_OK;
}

// ------------------------------------------------------------ (re)start
// Per rhs, by active[r]:
//   0: marked done, left untouched;
//   1: restart: r = convert(r_outer); rhat = r; p = r; x = 0; rho = ||r||^2;
//   3: as 1 but x is kept (a further segment of one inner solve whose
//      residual r_outer was recomputed in a higher precision);
//   2: reliable update: r = convert(r_outer), the true residual of the
//      current outer solution; x = 0; rhat and p are kept, rho = <rhat, r>,
//      and beta = (rho / rho_old)(alpha / omega) of the interrupted
//      iteration is set so that the p update that follows continues the
//      same Krylov recurrence (Sleijpen & van der Vorst's reliable updating).
// In both cases target2 = delta2 * ||r||^2.

template <int PO, int P, int PX>
__global__ void __launch_bounds__(kBlock) k_restart(Geom g, Vec r64, Vec r, Vec rhat, Vec p, Vec x, BiState *state,
                                                    double *partials, const int *active, const double *delta2)
{
    const SiteIdx q = site_idx(r.nrhs);
    BiState &S = state[q.r];
    const int mode = active[q.r];
    if (!mode) {
        if (q.sb == 0 && threadIdx.x == 0) S.done = 1;
        return;
    }
    using R = RT<P>;
    using RedT = typename RedType<R>::T;
    RedT red[3] = {RedT(0), RedT(0), RedT(0)};
    if (q.i < g.Vh) {
        cx<RT<PO>> a[12];
        SpinorIO<PO>::load(r64.rhs(q.r), g.stride, q.i, a);
        cx<R> v[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) v[k] = cconv<R>(a[k]);
        SpinorIO<P>::store_rounded(r.rhs(q.r), g.stride, q.i, v);
        cx<R> h[12];
        if (mode != 2) {
            st<P>(rhat, q.r, g.stride, q.i, v);
            st<P>(p, q.r, g.stride, q.i, v);
#pragma unroll
            for (int k = 0; k < 12; ++k) h[k] = v[k];
        } else {
            ld<P>(rhat, q.r, g.stride, q.i, h);
        }
        if (mode != 3) {
            cx<RT<PX>> z[12];
#pragma unroll
            for (int k = 0; k < 12; ++k) z[k] = {RT<PX>(0), RT<PX>(0)};
            SpinorIO<PX>::store(x.rhs(q.r), g.stride, q.i, z);
        }
        cx<R> d = {R(0), R(0)};
        R n = R(0);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            d = conjmad(h[k], v[k], d);
            n = fma(v[k].re, v[k].re, fma(v[k].im, v[k].im, n));
        }
        red[0] = d.re;
        red[1] = d.im;
        red[2] = n;
    }
    double tot[3];
    if (grid_sum<3>(red, partials + (size_t)q.r * q.nsb * kRedNV, &S.ticket[3], q.sb, q.nsb, tot) &&
        threadIdx.x == 0) {
        const double rr = tot[2];
        double bre = 0.0, bim = 0.0, ore = 0.0, oim = 0.0;
        if (mode == 2) {
            // beta = (rho_new / rho_old) (alpha / omega); without a usable
            // previous iteration the direction restarts from r (beta = 0)
            const double rho2 = S.rho_re * S.rho_re + S.rho_im * S.rho_im;
            const double om2 = S.omega_re * S.omega_re + S.omega_im * S.omega_im;
            if (rho2 > 0.0 && om2 > 0.0) {
                const double qre = (tot[0] * S.rho_re + tot[1] * S.rho_im) / rho2;
                const double qim = (tot[1] * S.rho_re - tot[0] * S.rho_im) / rho2;
                const double wre = (S.alpha_re * S.omega_re + S.alpha_im * S.omega_im) / om2;
                const double wim = (S.alpha_im * S.omega_re - S.alpha_re * S.omega_im) / om2;
                bre = qre * wre - qim * wim;
                bim = qre * wim + qim * wre;
                ore = S.omega_re;
                oim = S.omega_im;
            }
            S.rho_re = tot[0];
            S.rho_im = tot[1];
        } else {
            S.rho_re = rr;
            S.rho_im = 0.0;
        }
        S.rr = rr;
        S.target2 = delta2[q.r] * rr;
        S.alpha_re = S.alpha_im = 0.0;
        S.beta_re = bre;
        S.beta_im = bim;
        S.omega_re = ore;
        S.omega_im = oim;
        S.iters = 0;
        S.breakdown = 0;
        S.done = (rr > 0.0 && isfinite(rr)) ? 0 : 1;
    }
}

template <int PO>
static int restart_po(const Geom &g, const Vec &r64, const Vec &r, const Vec &rhat, const Vec &p, const Vec &x,
                      BiState *state, double *partials, const int *active, const double *delta2, cudaStream_t s)
{
    const int gr = grid_of(g, r.nrhs);
    if (r.prec == WL_F64 && x.prec == WL_F64)
        k_restart<PO, WL_F64, WL_F64><<<gr, kBlock, 0, s>>>(g, r64, r, rhat, p, x, state, partials, active, delta2);
    else if (r.prec == WL_F32 && x.prec == WL_F32)
        k_restart<PO, WL_F32, WL_F32><<<gr, kBlock, 0, s>>>(g, r64, r, rhat, p, x, state, partials, active, delta2);
    else if (r.prec == WL_F16 && x.prec == WL_F32)
        k_restart<PO, WL_F16, WL_F32><<<gr, kBlock, 0, s>>>(g, r64, r, rhat, p, x, state, partials, active, delta2);
    else {
        set_error("blas_restart: unsupported precision pair");
        return WL_ERR_ARG;
    }
    WL_CUDA_TRY(cudaGetLastError());
    note_launch(s);
    return WL_OK;
}

int blas_restart(const Geom &g, const Vec &r64, const Vec &r, const Vec &rhat, const Vec &p, const Vec &x,
                 BiState *state, double *partials, const int *active, const double *delta2, cudaStream_t s)
{
    if (r64.prec == WL_DF) return restart_po<WL_DF>(g, r64, r, rhat, p, x, state, partials, active, delta2, s);
    if (r64.prec == WL_F32) return restart_po<WL_F32>(g, r64, r, rhat, p, x, state, partials, active, delta2, s);
    return restart_po<WL_F64>(g, r64, r, rhat, p, x, state, partials, active, delta2, s);
}

// ----------------------------------------- x_outer += e  (rhs with active != 0)

template <int PO, int PX>
__global__ void __launch_bounds__(kBlock) k_accum(Geom g, Vec e, Vec x64, const int *active)
{
    const SiteIdx q = site_idx(x64.nrhs);
    if (!active[q.r] || q.i >= g.Vh) return;
    cx<RT<PX>> a[12];
    cx<RT<PO>> b[12];
    SpinorIO<PX>::load(e.rhs(q.r), g.stride, q.i, a);
    SpinorIO<PO>::load(x64.rhs(q.r), g.stride, q.i, b);
#pragma unroll
    for (int k = 0; k < 12; ++k) b[k] = b[k] + cconv<RT<PO>>(a[k]);
    SpinorIO<PO>::store(x64.rhs(q.r), g.stride, q.i, b);
}

int blas_accum(const Geom &g, const Vec &e, const Vec &x64, const int *active, cudaStream_t s)
{
    const int gr = grid_of(g, x64.nrhs);
    if (x64.prec == WL_DF) {
        if (e.prec == WL_F64) k_accum<WL_DF, WL_F64><<<gr, kBlock, 0, s>>>(g, e, x64, active);
        else k_accum<WL_DF, WL_F32><<<gr, kBlock, 0, s>>>(g, e, x64, active);
    } else {
        if (e.prec == WL_F64) k_accum<WL_F64, WL_F64><<<gr, kBlock, 0, s>>>(g, e, x64, active);
        else k_accum<WL_F64, WL_F32><<<gr, kBlock, 0, s>>>(g, e, x64, active);
    }
    WL_CUDA_TRY(cudaGetLastError());
    note_launch(s);
    return WL_OK;
}

// --------------------------------------------- out = x + a * y (outer prec)

template <int PO>
__global__ void __launch_bounds__(kBlock) k_xpay(Geom g, Vec x, double a, Vec y, Vec out)
{
    const SiteIdx q = site_idx(out.nrhs);
    if (q.i >= g.Vh) return;
    using R = RT<PO>;
    cx<R> xv[12], yv[12];
    SpinorIO<PO>::load(x.rhs(q.r), g.stride, q.i, xv);
    SpinorIO<PO>::load(y.rhs(q.r), g.stride, q.i, yv);
    const R c = Conv<R>::from(a);
#pragma unroll
    for (int k = 0; k < 12; ++k) xv[k] = xv[k] + c * yv[k];
    SpinorIO<PO>::store(out.rhs(q.r), g.stride, q.i, xv);
}

int blas_xpay(const Geom &g, const Vec &x, double a, const Vec &y, const Vec &out, cudaStream_t s)
{
    const int gr = grid_of(g, out.nrhs);
    if (out.prec == WL_DF) k_xpay<WL_DF><<<gr, kBlock, 0, s>>>(g, x, a, y, out);
    else if (out.prec == WL_F64) k_xpay<WL_F64><<<gr, kBlock, 0, s>>>(g, x, a, y, out);
    else { set_error("blas_xpay: outer precision only"); return WL_ERR_ARG; }
    WL_CUDA_TRY(cudaGetLastError());
    note_launch(s);
    return WL_OK;
}

// ------------------------------------------------------ squared norm (FP64)
// out[r] = ||a_r||^2; uses tickets[r].

template <int P>
__global__ void __launch_bounds__(kBlock) k_norm2(Geom g, Vec a, double *out, double *partials, unsigned *tickets)
{
    const SiteIdx q = site_idx(a.nrhs);
    using NT = typename NormT<RT<P>>::T;
    NT red[1] = {NT(0)};
    if (q.i < g.Vh) {
        cx<RT<P>> v[12];
        ld<P>(a, q.r, g.stride, q.i, v);
        NT n = 0;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            norm_acc(n, v[k].re);
            norm_acc(n, v[k].im);
        }
        red[0] = n;
    }
    double tot[1];
    if (grid_sum<1>(red, partials + (size_t)q.r * q.nsb * kRedNV, &tickets[q.r], q.sb, q.nsb, tot) &&
        threadIdx.x == 0)
        out[q.r] = tot[0];
}

int blas_norm2(const Geom &g, const Vec &a, double *out_dev, double *partials, unsigned *tickets, cudaStream_t s)
{
    const int gr = grid_of(g, a.nrhs);
    switch (a.prec) {
    case WL_F64: k_norm2<WL_F64><<<gr, kBlock, 0, s>>>(g, a, out_dev, partials, tickets); break;
    case WL_F32: k_norm2<WL_F32><<<gr, kBlock, 0, s>>>(g, a, out_dev, partials, tickets); break;
    case WL_F16: k_norm2<WL_F16><<<gr, kBlock, 0, s>>>(g, a, out_dev, partials, tickets); break;
    case WL_DF: k_norm2<WL_DF><<<gr, kBlock, 0, s>>>(g, a, out_dev, partials, tickets); break;
    }
    WL_CUDA_TRY(cudaGetLastError());
    note_launch(s);
    return WL_OK;
}

// ------------------------------------- out = sum_j c_j in_j (FP64, k <= 16)
// coefficients per rhs: c[r * k + j] (complex, re/im arrays on the device).

struct LinIn {
    const void *p[32];
};

// out = sum_{j<k} c_j in_j and, optionally, out2 = sum_{j<k2} c2_j in_j
// (k <= k2: the first k inputs are shared and read once).  Coefficients per
// rhs: c[r * k + j], c2[r * k2 + j]; real, or complex (CPLX: re, im pairs).
template <int PO, bool CPLX>
__global__ void __launch_bounds__(kBlock) k_lincomb(Geom g, LinIn in, int k, int k2, size_t rhs_bytes, int nrhs,
                                                    const double *c1, const double *c2, Vec out, Vec out2)
{
    using R = RT<PO>;
    const SiteIdx q = site_idx(nrhs);
    if (q.i >= g.Vh) return;
    cx<R> acc[12], acc2[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) acc[c] = acc2[c] = {R(0), R(0)};
    const int kmax = k > k2 ? k : k2;
    for (int j = 0; j < kmax; ++j) {
        cx<R> v[12];
        SpinorIO<PO>::load(static_cast<const char *>(in.p[j]) + (size_t)q.r * rhs_bytes, g.stride, q.i, v);
        if constexpr (CPLX) {
            if (j < k) {
                const double *w = c1 + 2 * ((size_t)q.r * k + j);
                const cx<R> z = {Conv<R>::from(w[0]), Conv<R>::from(w[1])};
#pragma unroll
                for (int c = 0; c < 12; ++c) acc[c] = cmad(z, v[c], acc[c]);
            }
            if (j < k2) {
                const double *w = c2 + 2 * ((size_t)q.r * k2 + j);
                const cx<R> z = {Conv<R>::from(w[0]), Conv<R>::from(w[1])};
#pragma unroll
                for (int c = 0; c < 12; ++c) acc2[c] = cmad(z, v[c], acc2[c]);
            }
        } else {
            if (j < k) {
                const R w = Conv<R>::from(c1[q.r * k + j]);
#pragma unroll
                for (int c = 0; c < 12; ++c) acc[c] = {fma(w, v[c].re, acc[c].re), fma(w, v[c].im, acc[c].im)};
            }
            if (j < k2) {
                const R w = Conv<R>::from(c2[q.r * k2 + j]);
#pragma unroll
                for (int c = 0; c < 12; ++c) acc2[c] = {fma(w, v[c].re, acc2[c].re), fma(w, v[c].im, acc2[c].im)};
            }
        }
    }
    if (k > 0) SpinorIO<PO>::store(out.rhs(q.r), g.stride, q.i, acc);
    if (k2 > 0) SpinorIO<PO>::store(out2.rhs(q.r), g.stride, q.i, acc2);
}

int blas_lincomb2(const Geom &g, const double *c1_dev, const Vec *const *in, int k, const Vec *out,
                  const double *c2_dev, int k2, const Vec *out2, cudaStream_t s, bool complex_coef)
{
    if (k < 0 || k2 < 0 || k + k2 < 1 || k > 32 || k2 > 32) { set_error("blas_lincomb: 1..32 inputs"); return WL_ERR_ARG; }
    LinIn li;
    const int kmax = k > k2 ? k : k2;
    for (int j = 0; j < kmax; ++j) li.p[j] = in[j]->ptr;
    const Vec &o = k > 0 ? *out : *out2;
    Vec o2 = k2 > 0 ? *out2 : o;
    const Vec o1 = k > 0 ? *out : o2;
    const int grid = grid_of(g, o.nrhs);
    if (o.prec == WL_DF && complex_coef)
        k_lincomb<WL_DF, true><<<grid, kBlock, 0, s>>>(g, li, k, k2, o.rhs_bytes, o.nrhs, c1_dev, c2_dev, o1, o2);
    else if (o.prec == WL_DF)
        k_lincomb<WL_DF, false><<<grid, kBlock, 0, s>>>(g, li, k, k2, o.rhs_bytes, o.nrhs, c1_dev, c2_dev, o1, o2);
    else if (o.prec == WL_F64 && complex_coef)
        k_lincomb<WL_F64, true><<<grid, kBlock, 0, s>>>(g, li, k, k2, o.rhs_bytes, o.nrhs, c1_dev, c2_dev, o1, o2);
    else if (o.prec == WL_F64)
        k_lincomb<WL_F64, false><<<grid, kBlock, 0, s>>>(g, li, k, k2, o.rhs_bytes, o.nrhs, c1_dev, c2_dev, o1, o2);
    else { set_error("blas_lincomb: outer precision only"); return WL_ERR_ARG; }
    WL_CUDA_TRY(cudaGetLastError());
    note_launch(s);
    return WL_OK;
}

// Initial guess and first residual of a mass in one pass over the stored
// solutions x_j and their y_j = D_eo D_oe x_j (j < k):
//   x = sum_j c_j x_j,   r = b_prec - x + sum_j d_j y_j   (d_j = kappa^2 c_j),
// which by linearity is b_prec - M_prec x without a hop.  Written as
// b_prec - x + ..., x is formed once and subtracted, not recombined from
// the x_j: 48 k + 24 FMAs per site and rhs instead of 72 k + 24 -- in FP64,
// whose FMA rate on GB300 is 1/57 of FP32's, that is the cost of the pass.
// in: x_0..x_{k-1}, y_0..y_{k-1}, b_prec.  Coefficients per rhs: c[r k + j],
// d[r k + j] (complex: re, im pairs).
template <int PO, bool CPLX>
__global__ void __launch_bounds__(kBlock) k_guess_residual(Geom g, LinIn in, int k, size_t rhs_bytes, int nrhs,
                                                           const double *c, const double *d, Vec xo, Vec ro)
{
    using R = RT<PO>;
    const SiteIdx q = site_idx(nrhs);
    if (q.i >= g.Vh) return;
    const size_t off = (size_t)q.r * rhs_bytes;
    cx<R> x[12], r[12], v[12];
#pragma unroll
    for (int e = 0; e < 12; ++e) x[e] = acc_zero<R>();
    for (int j = 0; j < k; ++j) {
        SpinorIO<PO>::load(static_cast<const char *>(in.p[j]) + off, g.stride, q.i, v);
        if constexpr (CPLX) {
            const double *w = c + 2 * ((size_t)q.r * k + j);
            const cx<R> z = {Conv<R>::from(w[0]), Conv<R>::from(w[1])};
#pragma unroll
            for (int e = 0; e < 12; ++e) x[e] = cmad(z, v[e], x[e]);
        } else {
            const R w = Conv<R>::from(c[(size_t)q.r * k + j]);
#pragma unroll
            for (int e = 0; e < 12; ++e) x[e] = {fma(w, v[e].re, x[e].re), fma(w, v[e].im, x[e].im)};
        }
    }
    SpinorIO<PO>::load(static_cast<const char *>(in.p[2 * k]) + off, g.stride, q.i, r);
#pragma unroll
    for (int e = 0; e < 12; ++e) r[e] = r[e] - x[e];
    for (int j = 0; j < k; ++j) {
        SpinorIO<PO>::load(static_cast<const char *>(in.p[k + j]) + off, g.stride, q.i, v);
        if constexpr (CPLX) {
            const double *w = d + 2 * ((size_t)q.r * k + j);
            const cx<R> z = {Conv<R>::from(w[0]), Conv<R>::from(w[1])};
#pragma unroll
            for (int e = 0; e < 12; ++e) r[e] = cmad(z, v[e], r[e]);
        } else {
            const R w = Conv<R>::from(d[(size_t)q.r * k + j]);
#pragma unroll
            for (int e = 0; e < 12; ++e) r[e] = {fma(w, v[e].re, r[e].re), fma(w, v[e].im, r[e].im)};
        }
    }
    SpinorIO<PO>::store(xo.rhs(q.r), g.stride, q.i, x);
    SpinorIO<PO>::store(ro.rhs(q.r), g.stride, q.i, r);
}

int blas_guess_residual(const Geom &g, const double *c_dev, const double *d_dev, const Vec *const *in, int k,
                        const Vec &x, const Vec &r, cudaStream_t s, bool complex_coef)
{
    if (k < 0 || k > 15) { set_error("blas_guess_residual: 0..15 earlier solutions"); return WL_ERR_ARG; }
    LinIn li;
    for (int j = 0; j < 2 * k + 1; ++j) li.p[j] = in[j]->ptr;
    const int grid = grid_of(g, x.nrhs);
#define WL_GR(PO, CP) k_guess_residual<PO, CP><<<grid, kBlock, 0, s>>>(g, li, k, x.rhs_bytes, x.nrhs, c_dev, d_dev, x, r)
    if (x.prec == WL_DF && complex_coef) WL_GR(WL_DF, true);
    else if (x.prec == WL_DF) WL_GR(WL_DF, false);
    else if (x.prec == WL_F64 && complex_coef) WL_GR(WL_F64, true);
    else if (x.prec == WL_F64) WL_GR(WL_F64, false);
    else { set_error("blas_guess_residual: outer precision only"); return WL_ERR_ARG; }
#undef WL_GR
    WL_CUDA_TRY(cudaGetLastError());
    note_launch(s);
    return WL_OK;
}

int blas_lincomb(const Geom &g, const double *cre_dev, const double *, const Vec *const *in, int k,
                 const Vec &out, cudaStream_t s)
{
    return blas_lincomb2(g, cre_dev, in, k, &out, nullptr, 0, nullptr, s);
}

// -------------------------------- inner products of canonical vectors
// Solution-space minimisation (Section 6.2.2) needs the Gram matrix of the
// solutions and their overlap with the source; those are formed once per
// solved mass on the canonical complex128 outputs.

struct DotIn {
    const double2 *p[16];
};

template <int N>
__global__ void __launch_bounds__(256) k_canon_dots(const double2 *a, DotIn in, size_t n, double *partials,
                                                    unsigned *ticket, double *out)
{
    double v[2 * N];
#pragma unroll
    for (int j = 0; j < 2 * N; ++j) v[j] = 0.0;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        const double2 y = a[k];
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const double2 x = in.p[j][k];
            v[2 * j] += x.x * y.x + x.y * y.y;      // Re conj(x) y
            v[2 * j + 1] += x.x * y.y - x.y * y.x;  // Im conj(x) y
        }
    }
    double tot[2 * N];
    if (grid_sum<2 * N>(v, partials, ticket, blockIdx.x, gridDim.x, tot) && threadIdx.x == 0)
        for (int j = 0; j < 2 * N; ++j) out[j] = tot[j];
}

template <int N>
static void launch_canon_dots(const double2 *a, const DotIn &in, size_t n, double *partials, unsigned *ticket,
                              double *out, cudaStream_t s)
{
    k_canon_dots<N><<<1024, 256, 0, s>>>(a, in, n, partials, ticket, out);
}

int canon_dots(const void *const *a, const void *const *in, int n, int nrhs, size_t n_complex, double *dots_dev,
               double *partials, unsigned *tickets, cudaStream_t s)
{
    if (n < 1 || n > 16 || nrhs < 1) { set_error("canon_dots: 1..16 vectors"); return WL_ERR_ARG; }
    for (int r = 0; r < nrhs; ++r) {
        DotIn di;
        for (int j = 0; j < n; ++j) di.p[j] = static_cast<const double2 *>(in[r * n + j]);
        const double2 *ar = static_cast<const double2 *>(a[r]);
        double *o = dots_dev + 2 * (size_t)n * r;
        // the reduction width is a template parameter: round n up to 4, 8 or 16
        // (unused slots read input 0 and are ignored)
        const int nn = n <= 4 ? 4 : n <= 8 ? 8 : 16;
        for (int j = n; j < nn; ++j) di.p[j] = di.p[0];
        double *tmp = partials + 2 * 16 * 1024;  // nn outputs before the first n are kept
        if (nn == 4) launch_canon_dots<4>(ar, di, n_complex, partials, tickets + r, tmp, s);
        else if (nn == 8) launch_canon_dots<8>(ar, di, n_complex, partials, tickets + r, tmp, s);
        else launch_canon_dots<16>(ar, di, n_complex, partials, tickets + r, tmp, s);
        WL_CUDA_TRY(cudaGetLastError());
        note_launch(s);
        WL_CUDA_TRY(cudaMemcpyAsync(o, tmp, sizeof(double) * 2 * n, cudaMemcpyDeviceToDevice, s));
    }
    return WL_OK;
}

// ------------------------------ even-odd reconstruction with its residual
// x_o = b_o + kappa * Dx (Dx = D_oe x_e from the last residual check) and
// r_o = b_o - x_o + kappa * Dx, the odd part of the full-lattice residual,
// reduced to norm2[r] = ||r_o||^2.

template <int PO>
__global__ void __launch_bounds__(kBlock) k_recon(Geom g, Vec bo, Vec dx, double kappa, Vec xo, double *norm2,
                                                  double *partials, unsigned *tickets)
{
    using R = RT<PO>;
    const SiteIdx q = site_idx(xo.nrhs);
    double red[1] = {0.0};
    if (q.i < g.Vh) {
        cx<R> b[12], d[12], x[12];
        SpinorIO<PO>::load(bo.rhs(q.r), g.stride, q.i, b);
        SpinorIO<PO>::load(dx.rhs(q.r), g.stride, q.i, d);
        const R k = Conv<R>::from(kappa);
        typename NormT<R>::T n = 0;
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            cx<R> ro;
            if constexpr (PO == WL_F64) {
                // x = b + kappa d in one rounding; its rounding error
                // ro = (b - x) + kappa d, with the product fused again
                // (the FP64 pipe bounds this pass: 4 operations per real
                // instead of 5)
                x[c] = {fma(k, d[c].re, b[c].re), fma(k, d[c].im, b[c].im)};
                ro = {fma(k, d[c].re, b[c].re - x[c].re), fma(k, d[c].im, b[c].im - x[c].im)};
            } else {
                const cx<R> kd = k * d[c];
                x[c] = b[c] + kd;
                ro = (b[c] - x[c]) + kd;
            }
            norm_acc(n, ro.re);
            norm_acc(n, ro.im);
        }
        SpinorIO<PO>::store(xo.rhs(q.r), g.stride, q.i, x);
        red[0] = (double)n;
    }
    double tot[1];
    if (grid_sum<1>(red, partials + (size_t)q.r * q.nsb * kRedNV, &tickets[q.r], q.sb, q.nsb, tot) &&
        threadIdx.x == 0)
        norm2[q.r] = tot[0];
}

int blas_recon(const Geom &g, const Vec &bo, const Vec &dx, double kappa, const Vec &xo, double *norm2_dev,
               double *partials, unsigned *tickets, cudaStream_t s)
{
    const int gr = grid_of(g, xo.nrhs);
    if (xo.prec == WL_DF) k_recon<WL_DF><<<gr, kBlock, 0, s>>>(g, bo, dx, kappa, xo, norm2_dev, partials, tickets);
    else if (xo.prec == WL_F64) k_recon<WL_F64><<<gr, kBlock, 0, s>>>(g, bo, dx, kappa, xo, norm2_dev, partials, tickets);
    else { set_error("blas_recon: outer precision only"); return WL_ERR_ARG; }
    WL_CUDA_TRY(cudaGetLastError());
    note_launch(s);
    return WL_OK;
}

// ------------------------------------------------------------- conversion

template <int PI, int PO>
__global__ void __launch_bounds__(kBlock) k_convert(Geom g, Vec in, Vec out)
{
    const SiteIdx q = site_idx(out.nrhs);
    if (q.i >= g.Vh) return;
    cx<RT<PI>> a[12];
    cx<RT<PO>> b[12];
    SpinorIO<PI>::load(in.rhs(q.r), g.stride, q.i, a);
#pragma unroll
    for (int k = 0; k < 12; ++k) b[k] = cconv<RT<PO>>(a[k]);
    SpinorIO<PO>::store(out.rhs(q.r), g.stride, q.i, b);
}

int blas_convert(const Geom &g, const Vec &in, const Vec &out, cudaStream_t s)
{
    const int gr = grid_of(g, out.nrhs);
#define WL_CONV(A, B) \
    if (in.prec == A && out.prec == B) { k_convert<A, B><<<gr, kBlock, 0, s>>>(g, in, out); WL_CUDA_TRY(cudaGetLastError()); note_launch(s); return WL_OK; }
    WL_CONV(WL_F64, WL_F64) WL_CONV(WL_F64, WL_F32) WL_CONV(WL_F64, WL_F16)
    WL_CONV(WL_F32, WL_F64) WL_CONV(WL_F32, WL_F32) WL_CONV(WL_F32, WL_F16)
    WL_CONV(WL_F16, WL_F64) WL_CONV(WL_F16, WL_F32) WL_CONV(WL_F16, WL_F16)
    WL_CONV(WL_DF, WL_F64) WL_CONV(WL_F64, WL_DF) WL_CONV(WL_DF, WL_F32) WL_CONV(WL_DF, WL_DF)
#undef WL_CONV
    set_error("blas_convert: bad precision");
    return WL_ERR_ARG;
}

}  // namespace wl
