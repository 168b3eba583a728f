// Multi-shift BiCGstab-M baseline (Section 6.1).  One Krylov space on the
// full-lattice unshifted system A = M_p(m_s) = (m_s + 4) - D/2 with
// m_s = min m_i; each shift sigma_i = m_i - m_s carries its own x^s, p^s and
// the scalar recurrences below (Jegerlehner's method, which the paper cites
// and does not print), written for van der Vorst's sign conventions:
//   after alpha_n, omega_n:  c = alpha_n beta_{n-1} / alpha_{n-1}
//     pi_{n+1} = (1 + c + alpha_n sigma) pi_n - c pi_{n-1}
//     alpha^s = alpha_n pi_n / pi_{n+1},   omega^s = omega_n / (1 + omega_n sigma)
//     x^s += alpha^s p^s + omega^s s_n / (pi_{n+1} lambda_n)
//     q^s  = p^s - (omega^s / alpha^s) (r_n / (pi_n lambda_n) - s_n / (pi_{n+1} lambda_n))
//   after r_{n+1}, beta_n:   lambda_{n+1} = lambda_n (1 + omega_n sigma)
//     beta^s = beta_n (pi_n / pi_{n+1})^2
//     p^s = r_{n+1} / (pi_{n+1} lambda_{n+1}) + beta^s q^s
// The p^s update is applied lazily: each shift stores q^s, and the next
// iteration's x/q kernel forms p^s from it and r on the fly (one read and
// one write of the shift vectors per iteration fewer).
// The shifted residual is r_{n+1} / (pi_{n+1} lambda_{n+1}); a shift whose
// residual is below tol ||b|| is frozen (Section 6.1).  The vectors and hops
// are FP64 or double-float (48-bit significands on the FP32 pipes); the
// scalar recurrences are FP64 either way;
// each full-lattice vector stored as its even and odd halves.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

namespace wl {

// BiCGstab-M breakdown threshold: |<rhat, r>| or |<rhat, v>| below 1e-12 of
// its Cauchy-Schwarz bound (squared here).
constexpr double kBreakdown2 = 1e-24;

struct ShiftState {
    double sigma;
    double pim_re, pim_im;     // pi_{n-1}
    double pi_re, pi_im;       // pi_n
    double pin_re, pin_im;     // pi_{n+1}
    double lam_re, lam_im;     // lambda_n
    // coefficients of the current iteration's vector kernels (complex)
    double cxp_re, cxp_im;     // alpha^s
    double cxs_re, cxs_im;     // omega^s / (pi_{n+1} lambda_n)
    double cqr_re, cqr_im;     // -(omega^s/alpha^s) / (pi_n lambda_n)
    double cqs_re, cqs_im;     // +(omega^s/alpha^s) / (pi_{n+1} lambda_n)
    double cpr_re, cpr_im;     // 1 / (pi_{n+1} lambda_{n+1})
    double bs_re, bs_im;       // beta^s
    int active;
    int frozen_at;
};

// Previous-iteration scalars of the unshifted recursion.
struct MState {
    double alpha_prev_re, alpha_prev_im;
    double beta_prev_re, beta_prev_im;
    double target2;            // freeze a shift when ||r||^2 / |pi lambda|^2 < target2
    int iters;
    int finished;              // set once the unshifted recursion has stopped
};

__device__ __forceinline__ cx<double> dc(double re, double im) { return {re, im}; }
__device__ __forceinline__ cx<double> cdiv(cx<double> a, cx<double> b)
{
    const double d = b.re * b.re + b.im * b.im;
    return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}

// After alpha_n and omega_n: pi_{n+1}, alpha^s, omega^s and the x/q coefficients.
__global__ void k_shift_a(ShiftState *sh, int ns, const BiState *bs, const MState *ms)
{
    const int k = threadIdx.x;
    if (k >= ns || bs->done || !sh[k].active) return;
    ShiftState &S = sh[k];
    const cx<double> al = dc(bs->alpha_re, bs->alpha_im), om = dc(bs->omega_re, bs->omega_im);
    const cx<double> alp = dc(ms->alpha_prev_re, ms->alpha_prev_im), bep = dc(ms->beta_prev_re, ms->beta_prev_im);
    const cx<double> pim = dc(S.pim_re, S.pim_im), pi = dc(S.pi_re, S.pi_im), lam = dc(S.lam_re, S.lam_im);
    const cx<double> c = cdiv(al * bep, alp);
    const cx<double> one = {1.0, 0.0};
    const cx<double> f = one + c + S.sigma * al;
    const cx<double> pin = f * pi - c * pim;
    const cx<double> as = cdiv(al * pi, pin);
    const cx<double> os = cdiv(om, one + S.sigma * om);
    const cx<double> pl = pi * lam, pnl = pin * lam;
    const cx<double> cxs = cdiv(os, pnl);
    const cx<double> oa = cdiv(os, as);
    const cx<double> cqr = cdiv(oa, pl);
    const cx<double> cqs = cdiv(oa, pnl);
    S.pin_re = pin.re; S.pin_im = pin.im;
    S.cxp_re = as.re; S.cxp_im = as.im;
    S.cxs_re = cxs.re; S.cxs_im = cxs.im;
    S.cqr_re = -cqr.re; S.cqr_im = -cqr.im;
    S.cqs_re = cqs.re; S.cqs_im = cqs.im;
}

// After beta_n and ||r_{n+1}||: lambda_{n+1}, beta^s, p coefficient, freezing;
// then roll pi and the previous alpha/beta forward.
__global__ void k_shift_b(ShiftState *sh, int ns, const BiState *bs, MState *ms)
{
    const int k = threadIdx.x;
    if (ms->finished) return;     // uniform: no shift updates after the last iteration
    __syncthreads();
    if (bs->breakdown) {
        if (k == 0) ms->finished = 1;
        return;
    }
    if (k < ns && sh[k].active) {
        ShiftState &S = sh[k];
        const cx<double> om = dc(bs->omega_re, bs->omega_im), be = dc(bs->beta_re, bs->beta_im);
        const cx<double> pi = dc(S.pi_re, S.pi_im), pin = dc(S.pin_re, S.pin_im), lam = dc(S.lam_re, S.lam_im);
        const cx<double> one = {1.0, 0.0};
        const cx<double> lamn = lam * (one + S.sigma * om);
        const cx<double> q = cdiv(pi, pin);
        const cx<double> bsig = be * (q * q);
        const cx<double> pl = pin * lamn;
        const cx<double> cpr = cdiv(one, pl);
        S.cpr_re = cpr.re; S.cpr_im = cpr.im;
        S.bs_re = bsig.re; S.bs_im = bsig.im;
        S.pim_re = S.pi_re; S.pim_im = S.pi_im;
        S.pi_re = pin.re; S.pi_im = pin.im;
        S.lam_re = lamn.re; S.lam_im = lamn.im;
        const double pl2 = pl.re * pl.re + pl.im * pl.im;
        if (bs->rr / pl2 < ms->target2) {
            S.active = 0;
            S.frozen_at = bs->iters;
        }
    }
    __syncthreads();
    if (k == 0) {
        ms->alpha_prev_re = bs->alpha_re; ms->alpha_prev_im = bs->alpha_im;
        ms->beta_prev_re = bs->beta_re; ms->beta_prev_im = bs->beta_im;
        if (bs->done) ms->finished = 1;
    }
}

struct ShiftVecs {
    void *x[2][32];   // [half][shift]
    void *p[2][32];
};

// Grid: 2 * nsb blocks (half = blockIdx.x / nsb).
struct FullIdx {
    int half, sb, i;
};
__device__ __forceinline__ FullIdx full_idx(int nsb)
{
    FullIdx f;
    f.half = blockIdx.x / nsb;
    f.sb = blockIdx.x % nsb;
    f.i = f.sb * blockDim.x + threadIdx.x;
    return f;
}

// complex scalar of the vector arithmetic type
template <typename R>
__device__ __forceinline__ cx<R> cs(double re, double im) { return {Conv<R>::from(re), Conv<R>::from(im)}; }

// One spin-colour component c of site i (layouts as SpinorIO: FP64 double2
// [12][stride], double-float float4 [12][stride]).  The vector kernels below
// stream component by component, so a thread holds a few complex numbers
// instead of whole spinors per shift, and the kernels run at full occupancy.
template <int P> struct CompIO;
template <> struct CompIO<WL_F64> {
    using R = double;
    static __device__ __forceinline__ cx<R> ld(const void *base, int stride, int c, int i)
    {
        const double2 t = static_cast<const double2 *>(base)[(size_t)c * stride + i];
        return {t.x, t.y};
    }
    static __device__ __forceinline__ void st(void *base, int stride, int c, int i, cx<R> v)
    {
        static_cast<double2 *>(base)[(size_t)c * stride + i] = make_double2(v.re, v.im);
    }
};
template <> struct CompIO<WL_DF> {
    using R = df;
    static __device__ __forceinline__ cx<R> ld(const void *base, int stride, int c, int i)
    {
        const float4 t = static_cast<const float4 *>(base)[(size_t)c * stride + i];
        return {df(t.x, t.y), df(t.z, t.w)};
    }
    static __device__ __forceinline__ void st(void *base, int stride, int c, int i, cx<R> v)
    {
        const df re = df_normalize(v.re), im = df_normalize(v.im);
        static_cast<float4 *>(base)[(size_t)c * stride + i] = make_float4(re.hi, re.lo, im.hi, im.lo);
    }
};

template <int P>
__global__ void __launch_bounds__(kBlock) k_m_s(Geom g, int nsb, Vec r, Vec v, Vec s, const BiState *st)
{
    using C = CompIO<P>;
    using R = typename PrecTraits<P>::R;
    const FullIdx f = full_idx(nsb);
    if (__ldcg(&st->done) || f.i >= g.Vh) return;
    const cx<R> al = cs<R>(__ldcg(&st->alpha_re), __ldcg(&st->alpha_im));
    const int h = f.half, i = f.i, str = g.stride;
#pragma unroll 4
    for (int c = 0; c < 12; ++c) C::st(s.rhs(h), str, c, i, C::ld(r.rhs(h), str, c, i) - al * C::ld(v.rhs(h), str, c, i));
}

// Shift updates, p^s = cpr r + beta^s q^s (previous iteration's
// coefficients; cpr = 1, beta^s = 0 at the start), then x^s and q^s;
// unshifted x += alpha p + omega s, r = s - omega t with <rhat, r> and
// ||r||^2 -> beta (last block).
template <int P>
__global__ void __launch_bounds__(kBlock) k_m_update(Geom g, int nsb, Vec x, Vec p, Vec s, Vec t, Vec r, Vec rhat,
                                                     ShiftVecs sv, const ShiftState *sh, int ns, BiState *st,
                                                     double *partials)
{
    using C = CompIO<P>;
    using R = typename PrecTraits<P>::R;
    static_assert(sizeof(cx<R>) == 16, "coefficient staging assumes 16-byte complex scalars");
    const FullIdx f = full_idx(nsb);
    BiState &S = *st;
    if (__ldcg(&S.done)) return;
    // the active shifts and their six coefficients, staged once per block
    __shared__ alignas(16) unsigned char sraw[32 * 6 * 16];
    __shared__ int sact[32];
    __shared__ int snact;
    cx<R> *sc = reinterpret_cast<cx<R> *>(sraw);
    if (threadIdx.x < ns) {
        const ShiftState &Q = sh[threadIdx.x];
        cx<R> *q = sc + 6 * threadIdx.x;
        q[0] = cs<R>(Q.cxp_re, Q.cxp_im);
        q[1] = cs<R>(Q.cxs_re, Q.cxs_im);
        q[2] = cs<R>(Q.cqr_re, Q.cqr_im);
        q[3] = cs<R>(Q.cqs_re, Q.cqs_im);
        q[4] = cs<R>(Q.cpr_re, Q.cpr_im);
        q[5] = cs<R>(Q.bs_re, Q.bs_im);
    }
    if (threadIdx.x == 0) {
        int n = 0;
        for (int k = 0; k < ns; ++k)
            if (sh[k].active) sact[n++] = k;
        snact = n;
    }
    __syncthreads();
    double red[3] = {0.0, 0.0, 0.0};
    if (f.i < g.Vh) {
        const int h = f.half, i = f.i, str = g.stride, nact = snact;
        const cx<R> al = cs<R>(__ldcg(&S.alpha_re), __ldcg(&S.alpha_im));
        const cx<R> om = cs<R>(__ldcg(&S.omega_re), __ldcg(&S.omega_im));
        cx<R> d = {R(0), R(0)};
        R n = R(0);
#pragma unroll 2
        for (int c = 0; c < 12; ++c) {
            const cx<R> sc_ = C::ld(s.rhs(h), str, c, i), rc = C::ld(r.rhs(h), str, c, i);
            for (int j = 0; j < nact; ++j) {
                const int k = sact[j];
                const cx<R> *q = sc + 6 * k;
                cx<R> xs = C::ld(sv.x[h][k], str, c, i);
                const cx<R> ps = C::ld(sv.p[h][k], str, c, i);
                const cx<R> pc = cmad(q[4], rc, q[5] * ps);
                xs = cmad(q[0], pc, cmad(q[1], sc_, xs));
                C::st(sv.x[h][k], str, c, i, xs);
                C::st(sv.p[h][k], str, c, i, cmad(q[2], rc, cmad(q[3], sc_, pc)));
            }
            C::st(x.rhs(h), str, c, i, cmad(al, C::ld(p.rhs(h), str, c, i), cmad(om, sc_, C::ld(x.rhs(h), str, c, i))));
            const cx<R> rn = sc_ - om * C::ld(t.rhs(h), str, c, i);
            C::st(r.rhs(h), str, c, i, rn);
            d = conjmad(C::ld(rhat.rhs(h), str, c, i), rn, d);
            n = fma(rn.re, rn.re, fma(rn.im, rn.im, n));
        }
        red[0] = to_double(d.re);
        red[1] = to_double(d.im);
        red[2] = to_double(n);
    }
    double tot[3];
    if (grid_sum<3>(red, partials, &S.ticket[2], blockIdx.x, 2 * nsb, tot) && threadIdx.x == 0) {
        const double r1re = tot[0], r1im = tot[1], rr = tot[2];
        S.iters += 1;
        S.rr = rr;
        const double ore = S.omega_re, oim = S.omega_im;
        const double rho2 = S.rho_re * S.rho_re + S.rho_im * S.rho_im;
        const double om2 = ore * ore + oim * oim;
        const double r12 = r1re * r1re + r1im * r1im;
        if (!isfinite(rr)) {
            S.breakdown = 1;
            S.done = 1;
        } else if (rr <= S.target2) {
            S.done = 1;
        } else if (!(rho2 > 0.0) || !(om2 > 0.0) || !(r12 > S.brk2 * S.rhat2 * rr)) {
            // the next alpha would be rho / <rhat, v> with rho lost in rounding
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

// p = r + beta (p - omega v)  (the shifted p^s follow in k_m_update).
template <int P>
__global__ void __launch_bounds__(kBlock) k_m_p(Geom g, int nsb, Vec r, Vec p, Vec v, const BiState *st)
{
    using C = CompIO<P>;
    using R = typename PrecTraits<P>::R;
    const FullIdx f = full_idx(nsb);
    if (f.i >= g.Vh || __ldcg(&st->done)) return;
    const int h = f.half, i = f.i, str = g.stride;
    const cx<R> be = cs<R>(__ldcg(&st->beta_re), __ldcg(&st->beta_im));
    const cx<R> om = cs<R>(__ldcg(&st->omega_re), __ldcg(&st->omega_im));
#pragma unroll 4
    for (int c = 0; c < 12; ++c) {
        const cx<R> pv = C::ld(p.rhs(h), str, c, i), vv = C::ld(v.rhs(h), str, c, i);
        C::st(p.rhs(h), str, c, i, C::ld(r.rhs(h), str, c, i) + be * (pv - om * vv));
    }
}

// Sums over n complex entries of canonical arrays: out = {Re <a, b>, Im <a, b>, ||a||^2}.
__global__ void k_m_dots(const double2 *a, const double2 *b, size_t n, double *partials, unsigned *ticket,
                         double *out)
{
    double v[3] = {0.0, 0.0, 0.0};
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        const double2 x = a[k], y = b[k];
        v[0] += x.x * y.x + x.y * y.y;
        v[1] += x.x * y.y - x.y * y.x;
        v[2] += x.x * x.x + x.y * x.y;
    }
    double tot[3];
    if (grid_sum<3>(v, partials, ticket, blockIdx.x, gridDim.x, tot) && threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) out[k] = tot[k];
}

// r = p = b.  rhat = b (dots == nullptr: rho = ||b||^2) or a given shadow
// residual (dots = {Re <rhat, b>, Im <rhat, b>, ||rhat||^2}).
__global__ void k_m_init(BiState *st, double bn2, const double *dots, double target2, double brk2)
{
    st->rho_re = dots ? dots[0] : bn2;
    st->rho_im = dots ? dots[1] : 0.0;
    st->rhat2 = dots ? dots[2] : bn2;
    st->brk2 = brk2;
    st->rr = bn2;
    st->target2 = target2;
    st->done = 0;
    st->breakdown = 0;
    st->iters = 0;
}

static Vec half_of(const Vec &v, int h)
{
    Vec o = v;
    o.ptr = v.rhs(h);
    o.nrhs = 1;
    return o;
}

}  // namespace wl

using namespace wl;

extern "C" int bicgstab_m_solve(wl_gauge *g, const void *b, void *const *x, const double *m0, int n_mass,
                                const wl_solver_params *p, wl_solver_stats *stats, void *stream)
{
    if (!g || !b || !x || !m0 || !stats || !p || n_mass < 1 || n_mass > 32) {
        set_error("bicgstab_m_solve: bad argument (1 <= n_mass <= 32)");
        return WL_ERR_ARG;
    }
    if (!(p->tol > 0) || p->max_iter < 1) { set_error("bicgstab_m_solve: bad parameters"); return WL_ERR_ARG; }
    // vectors and hops in FP64 or double-float (outer_prec)
    const int P = p->outer_prec;
    if (P != WL_F64 && P != WL_DF) { set_error("bicgstab_m_solve: outer_prec must be FP64 or double-float"); return WL_ERR_ARG; }
    if (!(g->prec_mask & P)) {
        set_error(P == WL_DF ? "bicgstab_m_solve: needs double-float links" : "bicgstab_m_solve: needs FP64 links");
        return WL_ERR_ARG;
    }
    for (int i = 0; i < n_mass; ++i) {
        if (!x[i]) { set_error("bicgstab_m_solve: NULL solution"); return WL_ERR_ARG; }
        if (!(2.0 * m0[i] + 8.0 > 0.0)) { set_error("bicgstab_m_solve: need 2 m0 + 8 > 0"); return WL_ERR_ARG; }
        for (int j = 0; j < i; ++j)
            if (m0[i] == m0[j]) { set_error("bicgstab_m_solve: masses must be distinct"); return WL_ERR_ARG; }
    }
    auto t0 = std::chrono::steady_clock::now();
    std::unique_lock<std::mutex> lock(g->mu);
    cudaStream_t s = as_stream(stream);
    const Geom &geo = g->lat->geom;
    const int nsb = site_blocks(geo);
    int is = 0;
    for (int i = 1; i < n_mass; ++i)
        if (m0[i] < m0[is]) is = i;
    const double ms = m0[is];
    const int ns = n_mass - 1;

    // full-lattice vectors: 2 halves each
    Vec bv, xv, r, rhat, pv, v, sv, t;
    WL_TRY(make_vec(g, "bm_b", P, 2, &bv));
    WL_TRY(make_vec(g, "bm_x", P, 2, &xv));
    WL_TRY(make_vec(g, "bm_r", P, 2, &r));
    WL_TRY(make_vec(g, "bm_rhat", P, 2, &rhat));
    WL_TRY(make_vec(g, "bm_p", P, 2, &pv));
    WL_TRY(make_vec(g, "bm_v", P, 2, &v));
    WL_TRY(make_vec(g, "bm_s", P, 2, &sv));
    WL_TRY(make_vec(g, "bm_t", P, 2, &t));
    std::vector<Vec> xs(ns), ps(ns);
    ShiftVecs shv;
    std::vector<int> shift_mass(ns);
    for (int k = 0, i = 0; i < n_mass; ++i) {
        if (i == is) continue;
        WL_TRY(make_vec(g, "bm_xs" + std::to_string(k), P, 2, &xs[k]));
        WL_TRY(make_vec(g, "bm_ps" + std::to_string(k), P, 2, &ps[k]));
        for (int h = 0; h < 2; ++h) {
            shv.x[h][k] = xs[k].rhs(h);
            shv.p[h][k] = ps[k].rhs(h);
        }
        shift_mass[k] = i;
        ++k;
    }
    void *pst;
    WL_TRY(g->ws.get("bm_state", sizeof(BiState) + sizeof(MState) + sizeof(ShiftState) * 32 + 64, &pst));
    BiState *st = static_cast<BiState *>(pst);
    MState *mst = reinterpret_cast<MState *>(static_cast<char *>(pst) + sizeof(BiState));
    ShiftState *sh = reinterpret_cast<ShiftState *>(static_cast<char *>(pst) + sizeof(BiState) + sizeof(MState));
    void *ppart;
    WL_TRY(g->ws.get("bm_partials", sizeof(double) * 2 * nsb * kRedNV, &ppart));
    double *partials = static_cast<double *>(ppart);
    void *pn;
    WL_TRY(g->ws.get("bm_norm", sizeof(double) * 8 + sizeof(unsigned) * 4, &pn));
    double *d_norm = static_cast<double *>(pn);            // ||b_e||^2, ||b_o||^2, then rhat dots
    unsigned *d_ticket = reinterpret_cast<unsigned *>(d_norm + 8);

    // import b; ||b||^2
    const void *bc[1] = {b};
    Vec be = half_of(bv, 0), bo = half_of(bv, 1);
    WL_TRY(import_full(geo, bc, be, bo, s));
    WL_CUDA_TRY(cudaMemsetAsync(pn, 0, sizeof(double) * 8 + sizeof(unsigned) * 4, s));
    WL_TRY(blas_norm2(geo, be, d_norm, partials, d_ticket, s));
    WL_TRY(blas_norm2(geo, bo, d_norm + 1, partials, d_ticket + 1, s));
    double hn[2];
    WL_CUDA_TRY(cudaMemcpyAsync(hn, d_norm, sizeof(hn), cudaMemcpyDeviceToHost, s));
    WL_CUDA_TRY(cudaStreamSynchronize(s));
    const double bn2 = hn[0] + hn[1], bnorm = std::sqrt(bn2);

    // initial state: x = 0, r = rhat = p = b; x^s = 0, p^s = b
    const size_t vb = bv.rhs_bytes * 2;
    WL_CUDA_TRY(cudaMemsetAsync(xv.ptr, 0, vb, s));
    WL_CUDA_TRY(cudaMemcpyAsync(r.ptr, bv.ptr, vb, cudaMemcpyDeviceToDevice, s));
    double *d_dots = nullptr;
    if (p->shadow) {
        // given shadow residual: rho_0 = <rhat, b> must not vanish
        const void *sc[1] = {p->shadow};
        WL_TRY(import_full(geo, sc, half_of(rhat, 0), half_of(rhat, 1), s));
        void *pd;
        WL_TRY(g->ws.get("bm_dots_partials", sizeof(double) * 3 * 1024, &pd));
        d_dots = d_norm + 4;
        k_m_dots<<<1024, 256, 0, s>>>(static_cast<const double2 *>(p->shadow), static_cast<const double2 *>(b),
                                      (size_t)geo.Vh * 2 * 12, static_cast<double *>(pd), d_ticket + 2, d_dots);
        WL_CUDA_TRY(cudaGetLastError());
        note_launch(s);
        double hd[3];
        WL_CUDA_TRY(cudaMemcpyAsync(hd, d_dots, sizeof(hd), cudaMemcpyDeviceToHost, s));
        WL_CUDA_TRY(cudaStreamSynchronize(s));
        if (!(hd[0] * hd[0] + hd[1] * hd[1] > kBreakdown2 * hd[2] * bn2)) {
            set_error("bicgstab_m_solve: shadow residual (numerically) orthogonal to b");
            return WL_ERR_ARG;
        }
    } else {
        WL_CUDA_TRY(cudaMemcpyAsync(rhat.ptr, bv.ptr, vb, cudaMemcpyDeviceToDevice, s));
    }
    WL_CUDA_TRY(cudaMemcpyAsync(pv.ptr, bv.ptr, vb, cudaMemcpyDeviceToDevice, s));
    for (int k = 0; k < ns; ++k) {
        WL_CUDA_TRY(cudaMemsetAsync(xs[k].ptr, 0, vb, s));
        WL_CUDA_TRY(cudaMemcpyAsync(ps[k].ptr, bv.ptr, vb, cudaMemcpyDeviceToDevice, s));
    }
    std::vector<ShiftState> hsh(ns);
    for (int k = 0; k < ns; ++k) {
        std::memset(&hsh[k], 0, sizeof(ShiftState));
        hsh[k].sigma = m0[shift_mass[k]] - ms;
        hsh[k].pim_re = hsh[k].pi_re = hsh[k].lam_re = 1.0;
        hsh[k].cpr_re = 1.0;   // p^s_0 = r_0 = b (with beta^s = 0 and q^s = b stored)
        hsh[k].active = 1;
        hsh[k].frozen_at = -1;
    }
    MState hm;
    std::memset(&hm, 0, sizeof(hm));
    hm.alpha_prev_re = 1.0;
    const double tol = p->tol;
    hm.target2 = (tol * bnorm) * (tol * bnorm);
    WL_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(BiState), s));
    WL_CUDA_TRY(cudaMemcpyAsync(mst, &hm, sizeof(MState), cudaMemcpyHostToDevice, s));
    if (ns) WL_CUDA_TRY(cudaMemcpyAsync(sh, hsh.data(), sizeof(ShiftState) * ns, cudaMemcpyHostToDevice, s));
    // iterate the unshifted system to half the tolerance (iterated/true gap)
    k_m_init<<<1, 1, 0, s>>>(st, bn2, d_dots, 0.25 * hm.target2, kBreakdown2);
    note_launch(s);
    WL_CUDA_TRY(cudaStreamSynchronize(s));

    const double a1 = ms + 4.0;
    auto iteration = [&](cudaStream_t q) -> int {
        Vec pe = half_of(pv, 0), po = half_of(pv, 1), ve = half_of(v, 0), vo = half_of(v, 1);
        Vec se = half_of(sv, 0), so = half_of(sv, 1), te = half_of(t, 0), to = half_of(t, 1);
        Vec rhe = half_of(rhat, 0), rho = half_of(rhat, 1);
        // v = A p, <rhat, v> -> alpha
        WL_TRY(hop_reduce(g, 0, po, pe, a1, ve, rhe, -0.5, nullptr, WL_EVEN, 0, st, partials, 0, 2 * nsb, q));
        WL_TRY(hop_reduce(g, 0, pe, po, a1, vo, rho, -0.5, nullptr, WL_ODD, 0, st, partials, nsb, 2 * nsb, q));
        if (P == WL_DF) k_m_s<WL_DF><<<2 * nsb, kBlock, 0, q>>>(geo, nsb, r, v, sv, st);
        else k_m_s<WL_F64><<<2 * nsb, kBlock, 0, q>>>(geo, nsb, r, v, sv, st);
        note_launch(q);
        // t = A s, <t,s>, <t,t> -> omega
        WL_TRY(hop_reduce(g, 1, so, se, a1, te, rhe, -0.5, nullptr, WL_EVEN, 0, st, partials, 0, 2 * nsb, q));
        WL_TRY(hop_reduce(g, 1, se, so, a1, to, rho, -0.5, nullptr, WL_ODD, 0, st, partials, nsb, 2 * nsb, q));
        if (ns) {
            k_shift_a<<<1, 32, 0, q>>>(sh, ns, st, mst);
            note_launch(q);
        }
        if (P == WL_DF)
            k_m_update<WL_DF><<<2 * nsb, kBlock, 0, q>>>(geo, nsb, xv, pv, sv, t, r, rhat, shv, sh, ns, st, partials);
        else
            k_m_update<WL_F64><<<2 * nsb, kBlock, 0, q>>>(geo, nsb, xv, pv, sv, t, r, rhat, shv, sh, ns, st, partials);
        k_shift_b<<<1, 32, 0, q>>>(sh, ns, st, mst);
        if (P == WL_DF) k_m_p<WL_DF><<<2 * nsb, kBlock, 0, q>>>(geo, nsb, r, pv, v, st);
        else k_m_p<WL_F64><<<2 * nsb, kBlock, 0, q>>>(geo, nsb, r, pv, v, st);
        note_launch(q);
        note_launch(q);
        note_launch(q);
        WL_CUDA_TRY(cudaGetLastError());
        return WL_OK;
    };

    // graph-captured blocks of iterations, as in the single-mass solver
    const int K = p->mode == WL_MODE_GRAPH ? std::max(1, p->graph_iters) : 1;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;
    size_t graph_nodes = 0;
    if (p->mode == WL_MODE_GRAPH) {
        WL_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        int status = WL_OK;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            for (int k = 0; k < K && status == WL_OK; ++k) status = iteration(cap);
            e = cudaStreamEndCapture(cap, &graph);
        }
        if (e == cudaSuccess && status == WL_OK) e = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) {
            cudaGraphGetNodes(graph, nullptr, &graph_nodes);
            cudaGraphDestroy(graph);
        }
        if (e != cudaSuccess || status != WL_OK) {
            cudaStreamDestroy(cap);
            if (status != WL_OK) return status;
            set_error(std::string("bicgstab_m_solve graph: ") + cudaGetErrorString(e));
            return WL_ERR_CUDA;
        }
    }
    BiState hs;
    int done_iters = 0, status = WL_OK;
    for (;;) {
        if (exec) {
            cudaError_t e = cudaGraphLaunch(exec, s);
            if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); status = WL_ERR_CUDA; break; }
            add_launches((long long)graph_nodes);
        } else {
            status = iteration(s);
            if (status != WL_OK) break;
        }
        done_iters += K;
        cudaError_t e = cudaMemcpyAsync(&hs, st, sizeof(BiState), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); status = WL_ERR_CUDA; break; }
        if (hs.done || done_iters >= p->max_iter) break;
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (cap) cudaStreamDestroy(cap);
    if (status != WL_OK) return status;
    if (ns) WL_CUDA_TRY(cudaMemcpy(hsh.data(), sh, sizeof(ShiftState) * ns, cudaMemcpyDeviceToHost));
    const double unshifted_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();

    // outputs in kappa form x_i = (m_i + 4) psi_i, true residuals in the
    // vector precision; a mass still above tol is polished by single-mass
    // BiCGstab.
    Vec scaled;
    WL_TRY(make_vec(g, "bm_out", P, 2, &scaled));
    void *pc;
    WL_TRY(g->ws.get("bm_coef", sizeof(double) * 2, &pc));
    double *d_coef = static_cast<double *>(pc);
    int worst = hs.breakdown ? WL_ERR_BREAKDOWN : hs.done ? WL_OK : WL_ERR_NOCONV;
    std::vector<int> polish;
    for (int i = 0; i < n_mass; ++i) {
        std::memset(&stats[i], 0, sizeof(wl_solver_stats));
        stats[i].mass = m0[i];
        const Vec *src = &xv;
        int it = hs.iters;
        if (i != is) {
            int k = 0;
            while (shift_mass[k] != i) ++k;
            src = &xs[k];
            it = hsh[k].frozen_at >= 0 ? hsh[k].frozen_at : hs.iters;
        }
        const double c[2] = {m0[i] + 4.0, 0.0};
        WL_CUDA_TRY(cudaMemcpyAsync(d_coef, c, sizeof(c), cudaMemcpyHostToDevice, s));
        for (int h = 0; h < 2; ++h) {
            Vec in = half_of(*src, h), out = half_of(scaled, h);
            const Vec *ins[1] = {&in};
            WL_TRY(blas_lincomb(geo, d_coef, d_coef + 1, ins, 1, out, s));
        }
        void *xo[1] = {x[i]};
        WL_TRY(export_full(geo, half_of(scaled, 0), half_of(scaled, 1), xo, s));
        std::vector<double> rel;
        WL_TRY(full_relres(g, be, bo, half_of(scaled, 0), half_of(scaled, 1), 1.0 / (2.0 * m0[i] + 8.0), {bnorm}, rel, s));
        stats[i].iterations = it;
        stats[i].matvecs = 2 * it;
        stats[i].true_relres = rel[0];
        stats[i].status = worst;
        if (!(rel[0] <= tol)) polish.push_back(i);
    }
    WL_CUDA_TRY(cudaStreamSynchronize(s));
    const double total = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    lock.unlock();  // bicgstab_solve takes the handle lock itself
    for (int i = 0; i < n_mass; ++i) stats[i].seconds = total;
    for (int i : polish) {
        wl_solver_params pp = *p;
        // FP64 polish where the handle has FP64 links, else FP32 inside
        // double-float defect correction
        pp.inner_prec = (g->prec_mask & WL_F64) ? WL_F64 : WL_F32;
        pp.outer_prec = P;
        pp.eo = 1;
        wl_solver_stats pol;
        const int ps_ = bicgstab_solve(g, b, x[i], m0[i], &pp, &pol, stream);
        stats[i].restarts = pol.iterations;
        stats[i].true_relres = pol.true_relres;
        stats[i].status = ps_;
        if (ps_ != WL_OK) worst = ps_;
    }
    if (!polish.empty()) {
        const double t2 = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        for (int i = 0; i < n_mass; ++i) stats[i].seconds = t2;
    }
    if (hs.breakdown)
        set_error("bicgstab_m_solve: the shifted recurrences broke down after " + std::to_string(hs.iters) +
                  " iterations (<rhat, r> or <rhat, v> vanished; with rhat = b a point source this happens at "
                  "once: pass a shadow residual); unconverged masses were finished by single-mass BiCGstab");
    return checked_result(worst);
}
