// Backward of the multi-mass solve: gradients of a real loss L(x_1..x_n),
// x_i = M_k(m_i)^{-1} b, with respect to the links, the masses and the source.
//
// With g_i = dL/dRe x_i + i dL/dIm x_i (the complex gradient convention of
// PyTorch), dL = Re <lam_i, -dM x_i> + Re <lam_i, db> where lam_i solves the
// adjoint system M_k^dag lam_i = g_i.  M^dag = gamma5 M gamma5, so
// lam_i = gamma5 M^{-1} (gamma5 g_i): the adjoint solve reuses the forward
// solver.  Then (kappa form, M = 1 - kappa D):
//   links:  U_mu(n) -> exp(i h T) U_mu(n), T Hermitian traceless:
//           dL/dh = -kappa Im tr(T W_mu(n)),
//           W_mu(n) = s [ U x_{n+mu} (1 - gamma_mu) lam_n^dag - x_n (1 + gamma_mu) lam_{n+mu}^dag U^dag ]
//           (s = -1 across the antiperiodic time boundary), reported along
//           the generators T_a = lambda_a / 2 (Gell-Mann), 8 reals per link;
//   mass:   dM/dm0 = 2 kappa^2 D, so dL/dm0 = -Re <lam, 2 kappa^2 D x>;
//   source: dL/db = lam (same complex convention).
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

namespace wl {

using C = cx<double>;

__device__ __forceinline__ C cconj(C a) { return {a.re, -a.im}; }

// psi P for P = 1 - gamma_mu (plus = false) or 1 + gamma_mu (plus = true),
// psi a 3x4 colour x spin matrix (canonical [spin][colour] storage), through
// the Table 1 vectors: (psi P)_s = sum_k (psi v_k) v_k^dag[s].
__device__ void spin_project(const C *psi /*[4][3]*/, int mu, bool plus, C out[4][3])
{
    // (a1, c1, a2, c2) of the (1 - gamma) projector; phases 0:1 1:i 2:-1 3:-i
    const int a1 = mu >> 1, a2 = 1 - a1;
    int c1 = (0x0321 >> (4 * mu)) & 3, c2 = (0x0101 >> (4 * mu)) & 3;
    if (plus) {
        c1 = (c1 + 2) & 3;
        c2 = (c2 + 2) & 3;
    }
    auto ph = [](int c, C z) -> C {
        switch (c & 3) {
        case 0: return z;
        case 1: return {-z.im, z.re};
        case 2: return {-z.re, -z.im};
        default: return {z.im, -z.re};
        }
    };
    for (int c = 0; c < 3; ++c) {
        const C h1 = ph((4 - c1) & 3, psi[a1 * 3 + c]) + psi[3 * 3 + c];
        const C h2 = ph((4 - c2) & 3, psi[a2 * 3 + c]) + psi[2 * 3 + c];
        out[a1][c] = ph(c1, h1);
        out[3][c] = h1;
        out[a2][c] = ph(c2, h2);
        out[2][c] = h2;
    }
}

// One thread per (site n, direction mu): dU[mu][n][a] += -kappa Im tr(T_a W).
template <int PL>
__global__ void k_link_force(Geom g, const void *links_even, const void *links_odd, const double2 *x,
                             const double2 *lam, double kappa, double *dU)
{
    const size_t V = (size_t)g.Vh * 2;
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= 4 * V) return;
    const int mu = (int)(tid / V);
    const size_t n = tid % V;
    int c[4];
    size_t r = n;
    c[0] = (int)(r % g.X); r /= g.X;
    c[1] = (int)(r % g.Y); r /= g.Y;
    c[2] = (int)(r % g.Z);
    c[3] = (int)(r / g.Z);
    const int ext[4] = {g.X, g.Y, g.Z, g.T};
    const int par = (c[0] + c[1] + c[2] + c[3]) & 1;
    const int i = site_index(g, c[0], c[1], c[2], c[3]);
    int cm[4] = {c[0], c[1], c[2], c[3]};
    double sgn = 1.0;
    if (++cm[mu] == ext[mu]) {
        cm[mu] = 0;
        if (mu == 3 && g.antiperiodic) sgn = -1.0;
    }
    const size_t m = cm[0] + (size_t)g.X * (cm[1] + (size_t)g.Y * (cm[2] + (size_t)g.Z * cm[3]));
    // link U_mu(n) from the internal store (all three rows for FP64 and DF)
    cx<typename PrecTraits<PL>::R> ul[9];
    LinkIO<PL>::load(static_cast<const char *>(par ? links_odd : links_even) + (size_t)mu * link_dir_bytes(PL, g.stride),
                     g.stride, i, ul);
    C U[9];
    for (int k = 0; k < 9; ++k) U[k] = cconv<double>(ul[k]);
    C xm[12], xn[12], ln[12], lm[12];
    for (int k = 0; k < 12; ++k) {
        double2 t = x[m * 12 + k];
        xm[k] = {t.x, t.y};
        t = x[n * 12 + k];
        xn[k] = {t.x, t.y};
        t = lam[n * 12 + k];
        ln[k] = {t.x, t.y};
        t = lam[m * 12 + k];
        lm[k] = {t.x, t.y};
    }
    C Pm[4][3], Pp[4][3];
    spin_project(xm, mu, false, Pm);  // x_{n+mu} (1 - gamma_mu)
    spin_project(xn, mu, true, Pp);   // x_n (1 + gamma_mu)
    // A = U Pm (3x4)
    C A[4][3];
    for (int s = 0; s < 4; ++s)
        for (int a = 0; a < 3; ++a) {
            C t = {0.0, 0.0};
            for (int b = 0; b < 3; ++b) t = cmad(U[3 * a + b], Pm[s][b], t);
            A[s][a] = t;
        }
    // W = A lam_n^dag - (Pp lam_m^dag) U^dag
    C W[3][3], BL[3][3];
    for (int a = 0; a < 3; ++a)
        for (int cc = 0; cc < 3; ++cc) {
            C t1 = {0.0, 0.0}, t2 = {0.0, 0.0};
            for (int s = 0; s < 4; ++s) {
                t1 = cmad(A[s][a], cconj(ln[s * 3 + cc]), t1);
                t2 = cmad(Pp[s][a], cconj(lm[s * 3 + cc]), t2);
            }
            W[a][cc] = t1;
            BL[a][cc] = t2;
        }
    for (int a = 0; a < 3; ++a)
        for (int cc = 0; cc < 3; ++cc) {
            C t = {0.0, 0.0};
            for (int b = 0; b < 3; ++b) t = cmad(BL[a][b], cconj(U[3 * cc + b]), t);
            W[a][cc] = sgn * (W[a][cc] - t);
        }
    // Im tr(lambda_a W) / 2 for the eight Gell-Mann matrices
    double im[8];
    im[0] = (W[1][0] + W[0][1]).im;
    im[1] = (W[0][1].re - W[1][0].re);           // Im(-i W10 + i W01)
    im[2] = (W[0][0] - W[1][1]).im;
    im[3] = (W[2][0] + W[0][2]).im;
    im[4] = (W[0][2].re - W[2][0].re);           // Im(-i W20 + i W02)
    im[5] = (W[2][1] + W[1][2]).im;
    im[6] = (W[1][2].re - W[2][1].re);           // Im(-i W21 + i W12)
    im[7] = (W[0][0].im + W[1][1].im - 2.0 * W[2][2].im) / sqrt(3.0);
    double *out = dU + ((size_t)mu * V + n) * 8;
    for (int a = 0; a < 8; ++a) out[a] += -kappa * 0.5 * im[a];
}

// out = gamma5 in (canonical spinors): spins 2, 3 change sign.
__global__ void k_gamma5(const double2 *in, double2 *out, size_t V)
{
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= V * 12) return;
    const int s = (int)((k % 12) / 3);
    const double2 v = in[k];
    out[k] = s < 2 ? v : make_double2(-v.x, -v.y);
}

// acc += a (canonical)
__global__ void k_acc(const double2 *a, double2 *acc, size_t n)
{
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    acc[k] = make_double2(acc[k].x + a[k].x, acc[k].y + a[k].y);
}

// out = sum_k conj(a_k) b_k over n complex entries (FP64, deterministic)
__global__ void k_cdot(const double2 *a, const double2 *b, size_t n, double *partials, unsigned *ticket, double *out)
{
    double v[2] = {0.0, 0.0};
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        const double2 x = a[k], y = b[k];
        v[0] += x.x * y.x + x.y * y.y;
        v[1] += x.x * y.y - x.y * y.x;
    }
    double tot[2];
    if (grid_sum<2>(v, partials, ticket, blockIdx.x, gridDim.x, tot) && threadIdx.x == 0) {
        out[0] = tot[0];
        out[1] = tot[1];
    }
}

}  // namespace wl

using namespace wl;

extern "C" int wilson_solve_backward(wl_gauge *g, const void *b, const void *const *x, const void *const *gx,
                                     const double *m0, int n_mass, const wl_solver_params *p, double *dU,
                                     double *dm0, void *db, void *stream)
{
    if (!g || !b || !gx || !m0 || n_mass < 1 || !p || (!dU && !dm0 && !db)) {
        set_error("wilson_solve_backward: bad argument");
        return WL_ERR_ARG;
    }
    for (int i = 0; i < n_mass; ++i)
        if (!gx[i] || !(2.0 * m0[i] + 8.0 > 0.0)) {
            set_error("wilson_solve_backward: NULL gradient or 2 m0 + 8 <= 0");
            return WL_ERR_ARG;
        }
    const int PL = (g->prec_mask & WL_F64) ? WL_F64 : (g->prec_mask & WL_DF) ? WL_DF : 0;
    if (!PL) { set_error("wilson_solve_backward: needs FP64 or double-float links"); return WL_ERR_ARG; }
    cudaStream_t s = as_stream(stream);
    const Geom &geo = g->lat->geom;
    const size_t V = (size_t)geo.Vh * 2;
    const size_t vbytes = V * 12 * sizeof(double2);
    void *px, *plam, *ptmp, *pred;
    {
        std::lock_guard<std::mutex> lock(g->mu);
        WL_TRY(g->ws.get("bw_x", vbytes, &px));
        WL_TRY(g->ws.get("bw_lam", vbytes, &plam));
        WL_TRY(g->ws.get("bw_tmp", vbytes, &ptmp));
        WL_TRY(g->ws.get("bw_red", sizeof(double) * (2 * 1024 + 2) + 64, &pred));
    }
    double2 *bx = static_cast<double2 *>(px), *blam = static_cast<double2 *>(plam), *btmp = static_cast<double2 *>(ptmp);
    double *partials = static_cast<double *>(pred);
    double *d_dot = partials + 2 * 1024;
    unsigned *ticket = reinterpret_cast<unsigned *>(d_dot + 2);
    WL_CUDA_TRY(cudaMemsetAsync(ticket, 0, sizeof(unsigned), s));
    const int th = 256;
    const unsigned nb12 = (unsigned)((V * 12 + th - 1) / th);
    for (int i = 0; i < n_mass; ++i) {
        const double kappa = 1.0 / (2.0 * m0[i] + 8.0);
        wl_solver_stats st;
        // x_i: given, or re-solved
        const double2 *xi = static_cast<const double2 *>(x ? x[i] : nullptr);
        if (!xi) {
            WL_CUDA_TRY(cudaMemsetAsync(bx, 0, vbytes, s));
            const int rc = bicgstab_solve(g, b, bx, m0[i], p, &st, stream);
            if (rc != WL_OK) return rc;
            xi = bx;
        }
        // lam = gamma5 M^{-1} gamma5 g
        k_gamma5<<<nb12, th, 0, s>>>(static_cast<const double2 *>(gx[i]), btmp, V);
        WL_CUDA_TRY(cudaGetLastError());
        note_launch(s);
        WL_CUDA_TRY(cudaMemsetAsync(blam, 0, vbytes, s));
        const int rc = bicgstab_solve(g, btmp, blam, m0[i], p, &st, stream);
        if (rc != WL_OK) return rc;
        k_gamma5<<<nb12, th, 0, s>>>(blam, blam, V);
        WL_CUDA_TRY(cudaGetLastError());
        note_launch(s);
        if (dU) {
            const unsigned nbf = (unsigned)((4 * V + 127) / 128);
            if (PL == WL_F64)
                k_link_force<WL_F64><<<nbf, 128, 0, s>>>(geo, g->links[prec_index(WL_F64)][0],
                                                         g->links[prec_index(WL_F64)][1], xi, blam, kappa, dU);
            else
                k_link_force<WL_DF><<<nbf, 128, 0, s>>>(geo, g->links[prec_index(WL_DF)][0],
                                                        g->links[prec_index(WL_DF)][1], xi, blam, kappa, dU);
            WL_CUDA_TRY(cudaGetLastError());
            note_launch(s);
        }
        if (dm0) {
            // dL/dm0 = -Re <lam, 2 kappa^2 D x>
            WL_TRY(wilson_dslash(g, xi, btmp, kappa, PL, WL_OP_HOP, stream));
            k_cdot<<<1024, 256, 0, s>>>(blam, btmp, V * 12, partials, ticket, d_dot);
            WL_CUDA_TRY(cudaGetLastError());
            note_launch(s);
            double h[2];
            WL_CUDA_TRY(cudaMemcpyAsync(h, d_dot, sizeof(h), cudaMemcpyDeviceToHost, s));
            WL_CUDA_TRY(cudaStreamSynchronize(s));
            dm0[i] = -2.0 * kappa * kappa * h[0];
        }
        if (db) {
            k_acc<<<nb12, th, 0, s>>>(blam, static_cast<double2 *>(db), V * 12);
            WL_CUDA_TRY(cudaGetLastError());
            note_launch(s);
        }
    }
    WL_CUDA_TRY(cudaStreamSynchronize(s));
    return checked_result(WL_OK);
}
