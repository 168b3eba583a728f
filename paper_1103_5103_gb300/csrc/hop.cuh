// Wilson hop kernels D_eo / D_oe (Section 2, Eq. 4; Algorithm 1) for sm_103a.
// Device code shared by the per-precision translation units hop_*.cu.
//
// One thread per output site of one parity (the paper's granularity choice,
// Section 4), NB right-hand sides per thread sharing each link load.  Per
// direction the neighbour spinor is "shrunk" to two colour vectors with the
// Table 1 projector vectors, multiplied by the (12-real, row-2 rebuilt)
// link, and "expanded" back into the accumulator.  The projector entries
// are unit phases {+-1, +-i}, so shrink and expand are only adds and
// re/im swaps.  Epilogues fuse the xpay of M_prec and the BiCGstab inner
// products so that v = A p and t = A s are produced together with the
// scalars alpha and omega.
#pragma once

#include "internal.h"

namespace wl {

// Unit phase code: 0 -> 1, 1 -> i, 2 -> -1, 3 -> -i.
template <int C, typename R>
__device__ __forceinline__ cx<R> uphase(cx<R> z)
{
    if constexpr (C == 0) return z;
    else if constexpr (C == 1) return {-z.im, z.re};
    else if constexpr (C == 2) return {-z.re, -z.im};
    else return {z.im, -z.re};
}

// Table 1, forward transporter T_mu^+ (spin matrix 1 - gamma_mu):
// v1^dag = c1 at spin a1, 1 at spin 3;  v2^dag = c2 at spin a2, 1 at spin 2.
// The backward transporter T_mu^- (1 + gamma_mu) has c1, c2 negated.
template <int MU> struct Proj;
template <> struct Proj<0> { static constexpr int a1 = 0, c1 = 1, a2 = 1, c2 = 1; };  // (i,0,0,1) (0,i,1,0)
template <> struct Proj<1> { static constexpr int a1 = 0, c1 = 2, a2 = 1, c2 = 0; };  // (-1,0,0,1) (0,1,1,0)
template <> struct Proj<2> { static constexpr int a1 = 1, c1 = 3, a2 = 0, c2 = 1; };  // (0,-i,0,1) (i,0,1,0)
template <> struct Proj<3> { static constexpr int a1 = 1, c1 = 0, a2 = 0, c2 = 0; };  // (0,1,0,1) (1,0,1,0)

// acc += sc * L psi (1 -/+ gamma_MU) with L = u (ADJ = false) or u^dag.
// PLUS = 0 selects (1 - gamma_MU), PLUS = 1 selects (1 + gamma_MU).
// Spinor component k = 3*spin + colour.  sc carries the time-boundary sign
// and, for FP16 storage, the neighbour's per-site norm (psi then holds the
// unscaled halves): shrink and colour multiplication are linear, so the
// scale is applied once, in the multiply-adds of the expand, instead of to
// the 24 loaded values.  For sc = +-1 the fused multiply-add is exactly
// the add or subtract it replaces.
template <typename R>
__device__ __forceinline__ cx<R> cfma(R s, cx<R> z, cx<R> a)
{
    return {fma(s, z.re, a.re), fma(s, z.im, a.im)};
}

template <int MU, int PLUS, bool ADJ, typename R>
__device__ __forceinline__ void transport(cx<R> (&acc)[12], const cx<R> (&psi)[12], const cx<R> (&u)[9], R sc)
{
    constexpr int A1 = Proj<MU>::a1, A2 = Proj<MU>::a2;
    constexpr int C1 = (Proj<MU>::c1 + 2 * PLUS) & 3, C2 = (Proj<MU>::c2 + 2 * PLUS) & 3;
    constexpr int C1c = (4 - C1) & 3, C2c = (4 - C2) & 3;  // conjugate phases
    // shrink: h_k = psi v_k (v_k = conj(v_k^dag))
    cx<R> h1[3], h2[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        h1[c] = uphase<C1c>(psi[3 * A1 + c]) + psi[9 + c];
        h2[c] = uphase<C2c>(psi[3 * A2 + c]) + psi[6 + c];
    }
    // colour multiplication
    cx<R> w1[3], w2[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        cx<R> s1 = {R(0), R(0)}, s2 = {R(0), R(0)};
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            if constexpr (!ADJ) {
                s1 = cmad(u[3 * a + b], h1[b], s1);
                s2 = cmad(u[3 * a + b], h2[b], s2);
            } else {
                s1 = conjmad(u[3 * b + a], h1[b], s1);
                s2 = conjmad(u[3 * b + a], h2[b], s2);
            }
        }
        w1[a] = s1;
        w2[a] = s2;
    }
    // expand: res_s += sc w_k v_k^dag[s]
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        acc[3 * A1 + c] = cfma(sc, uphase<C1>(w1[c]), acc[3 * A1 + c]);
        acc[9 + c] = cfma(sc, w1[c], acc[9 + c]);
        acc[3 * A2 + c] = cfma(sc, uphase<C2>(w2[c]), acc[3 * A2 + c]);
        acc[6 + c] = cfma(sc, w2[c], acc[6 + c]);
    }
}

struct HopArgs {
    Geom g;
    int out_parity;
    int nrhs;
    int ngroups;                 // ceil(nrhs / NB)
    const void *in;              // rhs r at in + r*rhs_bytes
    size_t rhs_bytes;
    const void *links_out;       // links at the output parity (forward links)
    const void *links_in;        // links at the input parity (backward links)
    const int *skip;             // optional per-rhs flags: skip rhs r when skip[r * skip_stride] != 0
    int skip_stride;
};

__device__ __forceinline__ bool rhs_done(const HopArgs &a, int r)
{
    return a.skip != nullptr && __ldcg(a.skip + (size_t)r * a.skip_stride) != 0;
}

// Forward and backward neighbours of site i (coordinates c, first site of
// its x row rowbase) in direction MU, and the antiperiodic sign flips of the
// two hops.
template <int MU>
__device__ __forceinline__ void neighbours(const Geom &g, int i, const Coord &c, int rowbase, int &fwd, int &bwd,
                                           bool &sf, bool &sb)
{
    sf = false;
    sb = false;
    if constexpr (MU == 0) {
        const int xf = c.x + 1 == g.X ? 0 : c.x + 1;
        const int xb = c.x == 0 ? g.X - 1 : c.x - 1;
        fwd = rowbase + (xf >> 1);
        bwd = rowbase + (xb >> 1);
    } else if constexpr (MU == 1) {
        fwd = c.y + 1 == g.Y ? i - (g.Y - 1) * g.Xh : i + g.Xh;
        bwd = c.y == 0 ? i + (g.Y - 1) * g.Xh : i - g.Xh;
    } else if constexpr (MU == 2) {
        const int s = g.Xh * g.Y;
        fwd = c.z + 1 == g.Z ? i - (g.Z - 1) * s : i + s;
        bwd = c.z == 0 ? i + (g.Z - 1) * s : i - s;
    } else {
        const int s = g.Xh * g.Y * g.Z;
        const bool lastt = c.t + 1 == g.T, firstt = c.t == 0;
        fwd = lastt ? i - (g.T - 1) * s : i + s;
        bwd = firstt ? i + (g.T - 1) * s : i - s;
        if (g.antiperiodic) {
            sf = lastt;
            sb = firstt;
        }
    }
}

// Accumulate the eight transporters of site i for NB right-hand sides.
template <int P, bool DAG, int NB, int MU, bool CG = false>
__device__ __forceinline__ void hop_dir(const HopArgs &a, int i, const Coord &c, int rowbase, int r0,
                                        cx<typename PrecTraits<P>::R> (&acc)[NB][12])
{
    using R = typename PrecTraits<P>::R;
    const Geom &g = a.g;
    int fwd, bwd;
    bool sf, sb;  // antiperiodic sign flips
    neighbours<MU>(g, i, c, rowbase, fwd, bwd, sf, sb);
    const size_t dir_off = (size_t)MU * link_dir_bytes(P, g.stride);
    cx<R> u[9];
    // forward: U_mu(n) psi_{n+mu} (1 - gamma_mu)   [dagger: (1 + gamma_mu)]
    LinkIO<P>::load(static_cast<const char *>(a.links_out) + dir_off, g.stride, i, u);
#pragma unroll
    for (int r = 0; r < NB; ++r) {
        if (NB > 1 && r0 + r >= a.nrhs) break;
        cx<R> psi[12];
        const R n = SpinorIO<P>::template load_unscaled<CG>(
            static_cast<const char *>(a.in) + (size_t)(r0 + r) * a.rhs_bytes, g.stride, fwd, psi);
        transport<MU, DAG ? 1 : 0, false>(acc[r], psi, u, sf ? -n : n);
    }
    // backward: U_mu(n-mu)^dag psi_{n-mu} (1 + gamma_mu)   [dagger: (1 - gamma_mu)]
    LinkIO<P>::load(static_cast<const char *>(a.links_in) + dir_off, g.stride, bwd, u);
#pragma unroll
    for (int r = 0; r < NB; ++r) {
        if (NB > 1 && r0 + r >= a.nrhs) break;
        cx<R> psi[12];
        const R n = SpinorIO<P>::template load_unscaled<CG>(
            static_cast<const char *>(a.in) + (size_t)(r0 + r) * a.rhs_bytes, g.stride, bwd, psi);
        transport<MU, DAG ? 0 : 1, true>(acc[r], psi, u, sb ? -n : n);
    }
}

// ---------------------------------------------------------------- epilogues

// out = a1 * x1 + a2 * x2 + coef * acc  (x1, x2 optional), per rhs.
struct EpiStore {
    void *out;
    void *out_raw;      // optional: also store the bare hop result D in
    const void *x1;
    const void *x2;
    double a1;
    double a2;
    double coef;
    size_t rhs_bytes;
    static constexpr int NV = 0;
    template <int P, int NB>
    __device__ __forceinline__ void operator()(const HopArgs &a, int i, bool active, int r0,
                                               cx<typename PrecTraits<P>::R> (&acc)[NB][12]) const
    {
        using R = typename PrecTraits<P>::R;
        if (!active) return;
#pragma unroll
        for (int r = 0; r < NB; ++r) {
            const int rr = r0 + r;
            if (rr >= a.nrhs || rhs_done(a, rr)) continue;
            const size_t off = (size_t)rr * rhs_bytes;
            if (out_raw) SpinorIO<P>::store(static_cast<char *>(out_raw) + off, a.g.stride, i, acc[r]);
            cx<R> o[12];
            const R c = Conv<R>::from(coef);
#pragma unroll
            for (int k = 0; k < 12; ++k) o[k] = c * acc[r][k];
            if (x1) {
                cx<R> v[12];
                SpinorIO<P>::load(static_cast<const char *>(x1) + off, a.g.stride, i, v);
#pragma unroll
                for (int k = 0; k < 12; ++k) o[k] = o[k] + Conv<R>::from(a1) * v[k];
            }
            if (x2) {
                cx<R> v[12];
                SpinorIO<P>::load(static_cast<const char *>(x2) + off, a.g.stride, i, v);
#pragma unroll
                for (int k = 0; k < 12; ++k) o[k] = o[k] + Conv<R>::from(a2) * v[k];
            }
            SpinorIO<P>::store(static_cast<char *>(out) + off, a.g.stride, i, o);
        }
    }
};

// Solver epilogues (NB = 1, one rhs per block):
//   KIND 0: v = p + coef*acc, reduce <rhat, v>  -> alpha = rho / <rhat, v>
//   KIND 1: t = s + coef*acc, reduce <t, s>, <t, t>  -> omega = <t,s>/<t,t>
//   KIND 2: w = p + coef*acc, reduce ||w||^2  -> alpha = ||z||^2 / ||w||^2 (CG)
//   KIND 3: z = r + coef*acc (dagger hop), reduce ||z||^2 -> beta (CG)
template <int KIND>
struct EpiReduce {
    void *out;
    const void *xin;    // p (KIND 0) or s (KIND 1)
    const void *rhat;   // KIND 0 only
    double a1;
    double coef;
    const double *coef_dev;  // if set, the coefficient is read from here (graph replays across masses)
    int blk_off, blk_total;
    size_t rhs_bytes;
    BiState *st;
    double *partials;   // [rhs][block][kRedNV]
    static constexpr int NV = 3;
};

template <int P, bool DAG, int NB, bool CG = false>
__device__ __forceinline__ void hop_accumulate(const HopArgs &a, int i, int r0,
                                               cx<typename PrecTraits<P>::R> (&acc)[NB][12])
{
    const Geom &g = a.g;
    const Coord c = site_coord(g, i, a.out_parity);
    const int rowbase = i - (c.x >> 1);
    hop_dir<P, DAG, NB, 0, CG>(a, i, c, rowbase, r0, acc);
    hop_dir<P, DAG, NB, 1, CG>(a, i, c, rowbase, r0, acc);
    hop_dir<P, DAG, NB, 2, CG>(a, i, c, rowbase, r0, acc);
    hop_dir<P, DAG, NB, 3, CG>(a, i, c, rowbase, r0, acc);
}

// ------------------------------------------------------- rolled variant
// The same stencil with the eight transporters in a loop that is not
// unrolled: projector, link orientation and neighbour are selected per trip
// (warp-uniform), so the loop body is compiled once.  For the double-float
// type the unrolled kernel is about 8x larger than the instruction cache
// and stalls on instruction fetch; this variant keeps the body resident.

// Runtime unit phase, code as in uphase: 0 -> 1, 1 -> i, 2 -> -1, 3 -> -i.
template <typename R>
__device__ __forceinline__ cx<R> uphase_rt(int c, cx<R> z)
{
    R re = (c & 1) ? z.im : z.re;
    R im = (c & 1) ? z.re : z.im;
    if (c == 1 || c == 2) re = -re;
    if (c >= 2) im = -im;
    return {re, im};
}

template <int P, bool DAG>
__device__ __forceinline__ void hop_accumulate_rolled(const HopArgs &a, int i, cx<typename PrecTraits<P>::R> (&acc)[12])
{
    using R = typename PrecTraits<P>::R;
    const Geom &g = a.g;
    const Coord c = site_coord(g, i, a.out_parity);
    const int rowbase = i - (c.x >> 1);
    const int sy = g.Xh, sz = g.Xh * g.Y, st = g.Xh * g.Y * g.Z;
    // neighbour indices [mu][fwd, bwd] and time-boundary sign flips
    int nb[8];
    nb[0] = rowbase + ((c.x + 1 == g.X ? 0 : c.x + 1) >> 1);
    nb[1] = rowbase + ((c.x == 0 ? g.X - 1 : c.x - 1) >> 1);
    nb[2] = c.y + 1 == g.Y ? i - (g.Y - 1) * sy : i + sy;
    nb[3] = c.y == 0 ? i + (g.Y - 1) * sy : i - sy;
    nb[4] = c.z + 1 == g.Z ? i - (g.Z - 1) * sz : i + sz;
    nb[5] = c.z == 0 ? i + (g.Z - 1) * sz : i - sz;
    nb[6] = c.t + 1 == g.T ? i - (g.T - 1) * st : i + st;
    nb[7] = c.t == 0 ? i + (g.T - 1) * st : i - st;
    const bool neg_f = g.antiperiodic && c.t + 1 == g.T, neg_b = g.antiperiodic && c.t == 0;
#pragma unroll 1
    for (int d = 0; d < 8; ++d) {
        const int mu = d >> 1;
        const bool fwd = (d & 1) == 0;
        const int j = nb[d];
        const bool neg = mu == 3 && (fwd ? neg_f : neg_b);
        // Table 1 (see Proj): a1 in {0,1}, a2 = 1 - a1; phases of the (1 - gamma) projector
        const int a1 = mu >> 1;
        const int c1m = (0x0321 >> (4 * mu)) & 3;   // mu: 0->1, 1->2, 2->3, 3->0
        const int c2m = (0x0101 >> (4 * mu)) & 3;   // mu: 0->1, 1->0, 2->1, 3->0
        const bool plus = fwd == DAG;               // (1 + gamma) on backward hops (swapped for dagger)
        const int c1 = (c1m + (plus ? 2 : 0)) & 3, c2 = (c2m + (plus ? 2 : 0)) & 3;
        const int c1c = (4 - c1) & 3, c2c = (4 - c2) & 3;
        cx<R> u[9];
        const size_t dir_off = (size_t)mu * link_dir_bytes(P, g.stride);
        LinkIO<P>::load(static_cast<const char *>(fwd ? a.links_out : a.links_in) + dir_off, g.stride, fwd ? i : j, u);
        cx<R> psi[12];
        SpinorIO<P>::load(a.in, g.stride, j, psi);
        cx<R> h1[3], h2[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const cx<R> pa1 = a1 == 0 ? psi[k] : psi[3 + k];
            const cx<R> pa2 = a1 == 0 ? psi[3 + k] : psi[k];
            h1[k] = uphase_rt(c1c, pa1) + psi[9 + k];
            h2[k] = uphase_rt(c2c, pa2) + psi[6 + k];
        }
        cx<R> w1[3], w2[3];
        if (fwd) {
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                cx<R> s1 = {R(0), R(0)}, s2 = {R(0), R(0)};
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    s1 = cmad(u[3 * r + b], h1[b], s1);
                    s2 = cmad(u[3 * r + b], h2[b], s2);
                }
                w1[r] = s1;
                w2[r] = s2;
            }
        } else {
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                cx<R> s1 = {R(0), R(0)}, s2 = {R(0), R(0)};
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    s1 = conjmad(u[3 * b + r], h1[b], s1);
                    s2 = conjmad(u[3 * b + r], h2[b], s2);
                }
                w1[r] = s1;
                w2[r] = s2;
            }
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (neg) {
                w1[k] = {-w1[k].re, -w1[k].im};
                w2[k] = {-w2[k].re, -w2[k].im};
            }
            const cx<R> t1 = uphase_rt(c1, w1[k]), t2 = uphase_rt(c2, w2[k]);
            acc[k] = acc[k] + (a1 == 0 ? t1 : t2);
            acc[3 + k] = acc[3 + k] + (a1 == 0 ? t2 : t1);
            acc[6 + k] = acc[6 + k] + w2[k];
            acc[9 + k] = acc[9 + k] + w1[k];
        }
    }
}

// FP32 rolled variant with a one-direction software prefetch: the raw
// 128-bit words of the next transporter's spinor and link are requested
// before the current one is computed, doubling the loads in flight per
// thread at the same register budget class.
struct RawF32 {
    float4 psi[6];
    float4 u[3];
};

__device__ __forceinline__ void raw_load_f32(const HopArgs &a, int d, int i, const int (&nb)[8], RawF32 &r)
{
    const int mu = d >> 1;
    const bool fwd = (d & 1) == 0;
    const int j = nb[d];
    const float4 *pl = reinterpret_cast<const float4 *>(static_cast<const char *>(fwd ? a.links_out : a.links_in) +
                                                        (size_t)mu * link_dir_bytes(WL_F32, a.g.stride));
    const int li = fwd ? i : j;
#pragma unroll
    for (int k = 0; k < 3; ++k) r.u[k] = __ldg(pl + (size_t)k * a.g.stride + li);
    const float4 *ps = static_cast<const float4 *>(a.in);
#pragma unroll
    for (int k = 0; k < 6; ++k) r.psi[k] = __ldg(ps + (size_t)k * a.g.stride + j);
}

template <bool DAG>
__device__ __forceinline__ void hop_accumulate_prefetch_f32(const HopArgs &a, int i, cx<float> (&acc)[12])
{
    using R = float;
    const Geom &g = a.g;
    const Coord c = site_coord(g, i, a.out_parity);
    const int rowbase = i - (c.x >> 1);
    const int sy = g.Xh, sz = g.Xh * g.Y, st = g.Xh * g.Y * g.Z;
    int nb[8];
    nb[0] = rowbase + ((c.x + 1 == g.X ? 0 : c.x + 1) >> 1);
    nb[1] = rowbase + ((c.x == 0 ? g.X - 1 : c.x - 1) >> 1);
    nb[2] = c.y + 1 == g.Y ? i - (g.Y - 1) * sy : i + sy;
    nb[3] = c.y == 0 ? i + (g.Y - 1) * sy : i - sy;
    nb[4] = c.z + 1 == g.Z ? i - (g.Z - 1) * sz : i + sz;
    nb[5] = c.z == 0 ? i + (g.Z - 1) * sz : i - sz;
    nb[6] = c.t + 1 == g.T ? i - (g.T - 1) * st : i + st;
    nb[7] = c.t == 0 ? i + (g.T - 1) * st : i - st;
    const bool neg_f = g.antiperiodic && c.t + 1 == g.T, neg_b = g.antiperiodic && c.t == 0;
    RawF32 cur, nxt;
    raw_load_f32(a, 0, i, nb, cur);
#pragma unroll 1
    for (int d = 0; d < 8; ++d) {
        if (d < 7) raw_load_f32(a, d + 1, i, nb, nxt);
        const int mu = d >> 1;
        const bool fwd = (d & 1) == 0;
        const bool neg = mu == 3 && (fwd ? neg_f : neg_b);
        const int a1 = mu >> 1;
        const int c1m = (0x0321 >> (4 * mu)) & 3;
        const int c2m = (0x0101 >> (4 * mu)) & 3;
        const bool plus = fwd == DAG;
        const int c1 = (c1m + (plus ? 2 : 0)) & 3, c2 = (c2m + (plus ? 2 : 0)) & 3;
        const int c1c = (4 - c1) & 3, c2c = (4 - c2) & 3;
        cx<R> u[9], psi[12];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            u[2 * k] = {cur.u[k].x, cur.u[k].y};
            u[2 * k + 1] = {cur.u[k].z, cur.u[k].w};
        }
        reconstruct_row2(u);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            psi[2 * k] = {cur.psi[k].x, cur.psi[k].y};
            psi[2 * k + 1] = {cur.psi[k].z, cur.psi[k].w};
        }
        cx<R> h1[3], h2[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const cx<R> pa1 = a1 == 0 ? psi[k] : psi[3 + k];
            const cx<R> pa2 = a1 == 0 ? psi[3 + k] : psi[k];
            h1[k] = uphase_rt(c1c, pa1) + psi[9 + k];
            h2[k] = uphase_rt(c2c, pa2) + psi[6 + k];
        }
        cx<R> w1[3], w2[3];
        if (fwd) {
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                cx<R> s1 = {R(0), R(0)}, s2 = {R(0), R(0)};
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    s1 = cmad(u[3 * r + b], h1[b], s1);
                    s2 = cmad(u[3 * r + b], h2[b], s2);
                }
                w1[r] = s1;
                w2[r] = s2;
            }
        } else {
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                cx<R> s1 = {R(0), R(0)}, s2 = {R(0), R(0)};
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    s1 = conjmad(u[3 * b + r], h1[b], s1);
                    s2 = conjmad(u[3 * b + r], h2[b], s2);
                }
                w1[r] = s1;
                w2[r] = s2;
            }
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (neg) {
                w1[k] = {-w1[k].re, -w1[k].im};
                w2[k] = {-w2[k].re, -w2[k].im};
            }
            const cx<R> t1 = uphase_rt(c1, w1[k]), t2 = uphase_rt(c2, w2[k]);
            acc[k] = acc[k] + (a1 == 0 ? t1 : t2);
            acc[3 + k] = acc[3 + k] + (a1 == 0 ? t2 : t1);
            acc[6 + k] = acc[6 + k] + w2[k];
            acc[9 + k] = acc[9 + k] + w1[k];
        }
        if (d < 7) cur = nxt;
    }
}

template <bool DAG, int MINB>
__global__ void __launch_bounds__(128, MINB) k_hop_prefetch_f32(HopArgs a, EpiStore epi)
{
    const int r = blockIdx.x % a.ngroups;
    const int sb = blockIdx.x / a.ngroups;
    if (rhs_done(a, r)) return;
    const int i = sb * blockDim.x + threadIdx.x;
    if (i >= a.g.Vh) return;
    HopArgs b = a;
    b.in = static_cast<const char *>(a.in) + (size_t)r * a.rhs_bytes;
    cx<float> acc[1][12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[0][k] = acc_zero<float>();
    hop_accumulate_prefetch_f32<DAG>(b, i, acc[0]);
    epi.template operator()<WL_F32, 1>(a, i, true, r, acc);
}

template <bool DAG, int MINB>
void launch_k_hop_prefetch_f32(HopArgs a, const EpiStore &e, cudaStream_t s)
{
    a.ngroups = a.nrhs;
    const int nsb = (a.g.Vh + 127) / 128;
    k_hop_prefetch_f32<DAG, MINB><<<nsb * a.nrhs, 128, 0, s>>>(a, e);
}

// ------------------------------------------ asynchronous-copy FP32 variant
// The link and the NB neighbour spinors of direction d+1 are copied into
// shared memory with cp.async while direction d is computed from shared
// memory (two stages).  Loads in flight hold no registers, so a thread
// keeps a whole direction outstanding while it computes.  Each thread reads
// back only the slots it filled itself, so its own cp.async.wait_group is
// the only ordering needed (no block barrier).

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <int NB>
struct AsyncHop {
    static constexpr int F4 = 3 + 6 * NB;  // float4 per thread and stage: link, then NB spinors
    static constexpr int smem_bytes = 2 * F4 * 128 * 16;
};

struct AsyncCtx {
    int i, r0, nr;      // site, first rhs, rhs in this group
    int nb[8];          // neighbour per direction d = 2 mu + (0 forward, 1 backward)
    bool neg_f, neg_b;  // antiperiodic sign of the forward / backward t hop
};

template <int NB>
__device__ __forceinline__ void async_issue(const HopArgs &a, const AsyncCtx &c, float4 *stage, int d, int buf)
{
    const int mu = d >> 1;
    const bool fwd = (d & 1) == 0;
    const int j = c.nb[d];
    const float4 *lk = reinterpret_cast<const float4 *>(static_cast<const char *>(fwd ? a.links_out : a.links_in) +
                                                        (size_t)mu * link_dir_bytes(WL_F32, a.g.stride));
    float4 *st = stage + (size_t)buf * AsyncHop<NB>::F4 * 128 + threadIdx.x;
    const int li = fwd ? c.i : j;
#pragma unroll
    for (int k = 0; k < 3; ++k) cp_async16(st + k * 128, lk + (size_t)k * a.g.stride + li);
#pragma unroll
    for (int r = 0; r < NB; ++r) {
        if (r >= c.nr) break;
        const float4 *sp = reinterpret_cast<const float4 *>(static_cast<const char *>(a.in) +
                                                            (size_t)(c.r0 + r) * a.rhs_bytes);
#pragma unroll
        for (int k = 0; k < 6; ++k) cp_async16(st + (3 + 6 * r + k) * 128, sp + (size_t)k * a.g.stride + j);
    }
}

template <int D, bool DAG, int NB>
__device__ __forceinline__ void async_step(const HopArgs &a, const AsyncCtx &c, float4 *stage,
                                           cx<float> (&acc)[NB][12])
{
    if constexpr (D < 7) {
        async_issue<NB>(a, c, stage, D + 1, (D + 1) & 1);
        cp_async_commit();
        cp_async_wait<1>();
    } else {
        cp_async_wait<0>();
    }
    constexpr int MU = D >> 1;
    constexpr bool FWD = (D & 1) == 0;
    const float4 *st = stage + (size_t)(D & 1) * AsyncHop<NB>::F4 * 128 + threadIdx.x;
    cx<float> u[9];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float4 t = st[k * 128];
        u[2 * k] = {t.x, t.y};
        u[2 * k + 1] = {t.z, t.w};
    }
    reconstruct_row2(u);
#pragma unroll
    for (int r = 0; r < NB; ++r) {
        if (r >= c.nr) break;
        cx<float> psi[12];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float4 t = st[(3 + 6 * r + k) * 128];
            psi[2 * k] = {t.x, t.y};
            psi[2 * k + 1] = {t.z, t.w};
        }
        if constexpr (FWD)
            transport<MU, DAG ? 1 : 0, false>(acc[r], psi, u, MU == 3 && c.neg_f ? -1.f : 1.f);
        else
            transport<MU, DAG ? 0 : 1, true>(acc[r], psi, u, MU == 3 && c.neg_b ? -1.f : 1.f);
    }
}

// acc[r] += D in[r0 + r] at site i (active threads only), r < nr <= NB,
// through the two-stage shared-memory pipeline; stage holds
// AsyncHop<NB>::smem_bytes of dynamic shared memory.
template <bool DAG, int NB>
__device__ __forceinline__ void hop_accumulate_async(const HopArgs &a, int i, int r0, int nr, float4 *stage,
                                                     cx<float> (&acc)[NB][12])
{
    const Geom &g = a.g;
    AsyncCtx c;
    c.i = i;
    c.r0 = r0;
    c.nr = nr;
    const Coord q = site_coord(g, i, a.out_parity);
    const int rowbase = i - (q.x >> 1);
    const int sy = g.Xh, sz = g.Xh * g.Y, stt = g.Xh * g.Y * g.Z;
    c.nb[0] = rowbase + ((q.x + 1 == g.X ? 0 : q.x + 1) >> 1);
    c.nb[1] = rowbase + ((q.x == 0 ? g.X - 1 : q.x - 1) >> 1);
    c.nb[2] = q.y + 1 == g.Y ? i - (g.Y - 1) * sy : i + sy;
    c.nb[3] = q.y == 0 ? i + (g.Y - 1) * sy : i - sy;
    c.nb[4] = q.z + 1 == g.Z ? i - (g.Z - 1) * sz : i + sz;
    c.nb[5] = q.z == 0 ? i + (g.Z - 1) * sz : i - sz;
    c.nb[6] = q.t + 1 == g.T ? i - (g.T - 1) * stt : i + stt;
    c.nb[7] = q.t == 0 ? i + (g.T - 1) * stt : i - stt;
    c.neg_f = g.antiperiodic && q.t + 1 == g.T;
    c.neg_b = g.antiperiodic && q.t == 0;
    async_issue<NB>(a, c, stage, 0, 0);
    cp_async_commit();
    async_step<0, DAG, NB>(a, c, stage, acc);
    async_step<1, DAG, NB>(a, c, stage, acc);
    async_step<2, DAG, NB>(a, c, stage, acc);
    async_step<3, DAG, NB>(a, c, stage, acc);
    async_step<4, DAG, NB>(a, c, stage, acc);
    async_step<5, DAG, NB>(a, c, stage, acc);
    async_step<6, DAG, NB>(a, c, stage, acc);
    async_step<7, DAG, NB>(a, c, stage, acc);
}

template <bool DAG, int NB, int MINB>
__global__ void __launch_bounds__(128, MINB) k_hop_async(HopArgs a, EpiStore epi)
{
    extern __shared__ float4 stage[];  // [2][F4][128]
    const int grp = blockIdx.x % a.ngroups;
    const int sb = blockIdx.x / a.ngroups;
    const int r0 = grp * NB;
    const int nr = a.nrhs - r0 < NB ? a.nrhs - r0 : NB;
    if (a.skip) {
        bool all_done = true;
        for (int r = r0; r < r0 + nr; ++r) all_done &= rhs_done(a, r);
        if (all_done) return;   // uniform over the block
    }
    const int i = sb * blockDim.x + threadIdx.x;
    const bool active = i < a.g.Vh;
    cx<float> acc[NB][12];
#pragma unroll
    for (int r = 0; r < NB; ++r)
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[r][k] = acc_zero<float>();
    if (active) hop_accumulate_async<DAG, NB>(a, i, r0, nr, stage, acc);
    epi.template operator()<WL_F32, NB>(a, i, active, r0, acc);
}

template <bool DAG, int NB, int MINB>
void launch_k_hop_async(HopArgs a, const EpiStore &e, cudaStream_t s)
{
    constexpr int smem = AsyncHop<NB>::smem_bytes;
    static bool attr = false;  // the opt-in above 48 KB, once per instantiation
    if (!attr) {
        cudaFuncSetAttribute(k_hop_async<DAG, NB, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        attr = true;
    }
    a.ngroups = (a.nrhs + NB - 1) / NB;
    const int nsb = (a.g.Vh + 127) / 128;
    k_hop_async<DAG, NB, MINB><<<nsb * a.ngroups, 128, smem, s>>>(a, e);
}

template <int P, bool DAG, int MINB>
__global__ void __launch_bounds__(128, MINB) k_hop_rolled(HopArgs a, EpiStore epi)
{
    using R = typename PrecTraits<P>::R;
    const int r = blockIdx.x % a.ngroups;
    const int sb = blockIdx.x / a.ngroups;
    if (rhs_done(a, r)) return;
    const int i = sb * blockDim.x + threadIdx.x;
    if (i >= a.g.Vh) return;
    HopArgs b = a;
    b.in = static_cast<const char *>(a.in) + (size_t)r * a.rhs_bytes;
    cx<R> acc[1][12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[0][k] = acc_zero<R>();
    hop_accumulate_rolled<P, DAG>(b, i, acc[0]);
    epi.template operator()<P, 1>(a, i, true, r, acc);
}

template <int P, bool DAG, int NB, int MINB>
__global__ void __launch_bounds__(128, MINB) k_hop(HopArgs a, EpiStore epi)
{
    using R = typename PrecTraits<P>::R;
    const int grp = blockIdx.x % a.ngroups;
    const int sb = blockIdx.x / a.ngroups;
    const int r0 = grp * NB;
    if (a.skip) {
        bool all_done = true;
        for (int r = r0; r < r0 + NB && r < a.nrhs; ++r) all_done &= rhs_done(a, r);
        if (all_done) return;
    }
    const int i = sb * blockDim.x + threadIdx.x;
    if (i >= a.g.Vh) return;
    cx<R> acc[NB][12];
#pragma unroll
    for (int r = 0; r < NB; ++r)
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[r][k] = acc_zero<R>();
    hop_accumulate<P, DAG, NB>(a, i, r0, acc);
    epi.template operator()<P, NB>(a, i, true, r0, acc);
}

// Grid-stride form of k_hop: a fixed grid of blocks_per_sm x SM-count
// blocks, each looping over the (site block, rhs group) tiles.  Meant for
// the FP64 hop, which is bound by the FP64 pipe (1/57 of the FP32 rate on
// GB300) and needs only a few warps per SM to keep it busy: with a small
// grid it leaves most warp slots and issue cycles to kernels of another
// stream running at the same time (another batch's FP32/FP16 inner solve),
// instead of occupying the GPU for its whole duration.
template <int P, bool DAG, int NB, int MINB>
__global__ void __launch_bounds__(128, MINB) k_hop_gs(HopArgs a, EpiStore epi)
{
    using R = typename PrecTraits<P>::R;
    const int nsb = (a.g.Vh + 127) / 128;
    const int ntiles = nsb * a.ngroups;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int grp = t % a.ngroups;
        const int sb = t / a.ngroups;
        const int r0 = grp * NB;
        if (a.skip) {
            bool all_done = true;
            for (int r = r0; r < r0 + NB && r < a.nrhs; ++r) all_done &= rhs_done(a, r);
            if (all_done) continue;
        }
        const int i = sb * blockDim.x + threadIdx.x;
        if (i >= a.g.Vh) continue;
        cx<R> acc[NB][12];
#pragma unroll
        for (int r = 0; r < NB; ++r)
#pragma unroll
            for (int k = 0; k < 12; ++k) acc[r][k] = acc_zero<R>();
        hop_accumulate<P, DAG, NB>(a, i, r0, acc);
        epi.template operator()<P, NB>(a, i, true, r0, acc);
    }
}

// ------------------------------------------------ paired-site variant
// Two output sites per thread, i and i + 64 of a 128-site tile (64-thread
// blocks, one rhs per block), with every FP32 operation of the stencil done
// on the pair at once by the packed sm_100+ instructions (__ffma2_rn,
// __fadd2_rn, __fmul2_rn: one issue slot for two lanes of arithmetic).
// Direction and projector phases are uniform over the pair; links,
// neighbours, FP16 norms and time-boundary signs are per site, so no operand
// is a broadcast.  Element .x of every float2 belongs to site a, .y to b.
struct pcx {
    float2 re, im;
};

__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
// b - a, exact as a single rounding: fma(-1, a, b)
__device__ __forceinline__ float2 psub(float2 b, float2 a) { return __ffma2_rn(make_float2(-1.f, -1.f), a, b); }
__device__ __forceinline__ float2 pneg(float2 a) { return __fmul2_rn(make_float2(-1.f, -1.f), a); }

__device__ __forceinline__ pcx pair_of(cx<float> a, cx<float> b) { return {make_float2(a.re, b.re), make_float2(a.im, b.im)}; }

// b + z * phase C (phase codes as in uphase)
template <int C>
__device__ __forceinline__ pcx padd_phase(pcx z, pcx b)
{
    if constexpr (C == 0) return {padd(b.re, z.re), padd(b.im, z.im)};
    else if constexpr (C == 1) return {psub(b.re, z.im), padd(b.im, z.re)};   // i z = (-z.im, z.re)
    else if constexpr (C == 2) return {psub(b.re, z.re), psub(b.im, z.im)};
    else return {padd(b.re, z.im), psub(b.im, z.re)};                          // -i z = (z.im, -z.re)
}

// acc + s * phase_C(w) with the scale pair s and its negation ns
template <int C>
__device__ __forceinline__ pcx pexpand(float2 s, float2 ns, pcx w, pcx acc)
{
    if constexpr (C == 0) return {pfma(s, w.re, acc.re), pfma(s, w.im, acc.im)};
    else if constexpr (C == 1) return {pfma(ns, w.im, acc.re), pfma(s, w.re, acc.im)};
    else if constexpr (C == 2) return {pfma(ns, w.re, acc.re), pfma(ns, w.im, acc.im)};
    else return {pfma(s, w.im, acc.re), pfma(ns, w.re, acc.im)};
}

// Row 2 of a pair of SU(3) links from rows 0 and 1: u[6+c] = conj(r0 x r1)_c.
__device__ __forceinline__ void reconstruct_row2_pair(pcx (&u)[9])
{
    pcx n[3];   // negated row 0
#pragma unroll
    for (int c = 0; c < 3; ++c) n[c] = {pneg(u[c].re), pneg(u[c].im)};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
        // a = u[c1] u[3+c2] - u[c2] u[3+c1];  row 2 = (a.re, -a.im)
        const pcx p = u[c1], q = u[3 + c2], r = u[c2], t = u[3 + c1];
        const pcx np = n[c1], nr = n[c2];
        const float2 re = pfma(p.re, q.re, pfma(np.im, q.im, pfma(nr.re, t.re, pmul(r.im, t.im))));
        const float2 im = pfma(np.re, q.im, pfma(np.im, q.re, pfma(r.re, t.im, pmul(r.im, t.re))));
        u[6 + c] = {re, im};
    }
}

// acc += s psi (1 -/+ gamma_MU) L for the pair, as transport() per site.
template <int MU, int PLUS, bool ADJ>
__device__ __forceinline__ void transport_pair(pcx (&acc)[12], const pcx (&psi)[12], const pcx (&u)[9], float2 s)
{
    constexpr int A1 = Proj<MU>::a1, A2 = Proj<MU>::a2;
    constexpr int C1 = (Proj<MU>::c1 + 2 * PLUS) & 3, C2 = (Proj<MU>::c2 + 2 * PLUS) & 3;
    constexpr int C1c = (4 - C1) & 3, C2c = (4 - C2) & 3;
    pcx h1[3], h2[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        h1[c] = padd_phase<C1c>(psi[3 * A1 + c], psi[9 + c]);
        h2[c] = padd_phase<C2c>(psi[3 * A2 + c], psi[6 + c]);
    }
    // u h:        re = sum u.re h.re - u.im h.im,  im = sum u.re h.im + u.im h.re
    // u^dag h:    re = sum u.re h.re + u.im h.im,  im = sum u.re h.im - u.im h.re
    float2 n1[3], n2[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        n1[b] = pneg(ADJ ? h1[b].re : h1[b].im);
        n2[b] = pneg(ADJ ? h2[b].re : h2[b].im);
    }
    const float2 mz = make_float2(-0.f, -0.f);
    pcx w1[3], w2[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        pcx s1 = {mz, mz}, s2 = {mz, mz};
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const pcx ub = ADJ ? u[3 * b + a] : u[3 * a + b];
            if constexpr (!ADJ) {
                s1 = {pfma(ub.re, h1[b].re, pfma(ub.im, n1[b], s1.re)), pfma(ub.re, h1[b].im, pfma(ub.im, h1[b].re, s1.im))};
                s2 = {pfma(ub.re, h2[b].re, pfma(ub.im, n2[b], s2.re)), pfma(ub.re, h2[b].im, pfma(ub.im, h2[b].re, s2.im))};
            } else {
                s1 = {pfma(ub.re, h1[b].re, pfma(ub.im, h1[b].im, s1.re)), pfma(ub.re, h1[b].im, pfma(ub.im, n1[b], s1.im))};
                s2 = {pfma(ub.re, h2[b].re, pfma(ub.im, h2[b].im, s2.re)), pfma(ub.re, h2[b].im, pfma(ub.im, n2[b], s2.im))};
            }
        }
        w1[a] = s1;
        w2[a] = s2;
    }
    const float2 ns = pneg(s);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        acc[3 * A1 + c] = pexpand<C1>(s, ns, w1[c], acc[3 * A1 + c]);
        acc[9 + c] = pexpand<0>(s, ns, w1[c], acc[9 + c]);
        acc[3 * A2 + c] = pexpand<C2>(s, ns, w2[c], acc[3 * A2 + c]);
        acc[6 + c] = pexpand<0>(s, ns, w2[c], acc[6 + c]);
    }
}

// Site and neighbour data of one site of a pair.
struct PairSite {
    int i, rowbase;
    Coord c;
};

template <int P, bool DAG, int MU>
__device__ __forceinline__ void hop_dir_pair(const HopArgs &a, const PairSite &sa, const PairSite &sb, pcx (&acc)[12])
{
    using R = float;
    const Geom &g = a.g;
    int fa, ba, fb, bb;
    bool sfa, sba, sfb, sbb;
    neighbours<MU>(g, sa.i, sa.c, sa.rowbase, fa, ba, sfa, sba);
    neighbours<MU>(g, sb.i, sb.c, sb.rowbase, fb, bb, sfb, sbb);
    const size_t dir_off = (size_t)MU * link_dir_bytes(P, g.stride);
    const char *lo = static_cast<const char *>(a.links_out) + dir_off;
    const char *li = static_cast<const char *>(a.links_in) + dir_off;
    {
        cx<R> ua[9], ub[9], pa[12], pb[12];
        LinkIO<P>::load_rows(lo, g.stride, sa.i, ua);
        LinkIO<P>::load_rows(lo, g.stride, sb.i, ub);
        const R na = SpinorIO<P>::load_unscaled(a.in, g.stride, fa, pa);
        const R nb = SpinorIO<P>::load_unscaled(a.in, g.stride, fb, pb);
        pcx u[9], psi[12];
#pragma unroll
        for (int k = 0; k < 6; ++k) u[k] = pair_of(ua[k], ub[k]);
        reconstruct_row2_pair(u);
#pragma unroll
        for (int k = 0; k < 12; ++k) psi[k] = pair_of(pa[k], pb[k]);
        transport_pair<MU, DAG ? 1 : 0, false>(acc, psi, u, make_float2(sfa ? -na : na, sfb ? -nb : nb));
    }
    {
        cx<R> ua[9], ub[9], pa[12], pb[12];
        LinkIO<P>::load_rows(li, g.stride, ba, ua);
        LinkIO<P>::load_rows(li, g.stride, bb, ub);
        const R na = SpinorIO<P>::load_unscaled(a.in, g.stride, ba, pa);
        const R nb = SpinorIO<P>::load_unscaled(a.in, g.stride, bb, pb);
        pcx u[9], psi[12];
#pragma unroll
        for (int k = 0; k < 6; ++k) u[k] = pair_of(ua[k], ub[k]);
        reconstruct_row2_pair(u);
#pragma unroll
        for (int k = 0; k < 12; ++k) psi[k] = pair_of(pa[k], pb[k]);
        transport_pair<MU, DAG ? 0 : 1, true>(acc, psi, u, make_float2(sba ? -na : na, sbb ? -nb : nb));
    }
}

// D applied at sites ia and ib of one rhs (a.in already offset to it);
// the results in A (site a) and B (site b).
template <int P, bool DAG>
__device__ __forceinline__ void hop_accumulate_pair(const HopArgs &a, int ia, int ib, cx<float> (&A)[1][12],
                                                    cx<float> (&B)[1][12])
{
    PairSite sa, sb;
    sa.i = ia;
    sa.c = site_coord(a.g, ia, a.out_parity);
    sa.rowbase = ia - (sa.c.x >> 1);
    sb.i = ib;
    sb.c = site_coord(a.g, ib, a.out_parity);
    sb.rowbase = ib - (sb.c.x >> 1);
    const float2 mz = make_float2(-0.f, -0.f);
    pcx acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = {mz, mz};
    hop_dir_pair<P, DAG, 0>(a, sa, sb, acc);
    hop_dir_pair<P, DAG, 1>(a, sa, sb, acc);
    hop_dir_pair<P, DAG, 2>(a, sa, sb, acc);
    hop_dir_pair<P, DAG, 3>(a, sa, sb, acc);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        A[0][k] = {acc[k].re.x, acc[k].im.x};
        B[0][k] = {acc[k].re.y, acc[k].im.y};
    }
}

constexpr int kPairThreads = 64;   // threads per block; 2 x 64 = 128 sites per tile

template <int P, bool DAG, int MINB>
__global__ void __launch_bounds__(kPairThreads, MINB) k_hop_pair(HopArgs a, EpiStore epi)
{
    const int r = blockIdx.x % a.ngroups;
    const int sb = blockIdx.x / a.ngroups;
    if (rhs_done(a, r)) return;
    const int ia = sb * (2 * kPairThreads) + threadIdx.x;
    if (ia >= a.g.Vh) return;
    const int ib = ia + kPairThreads;
    const bool has_b = ib < a.g.Vh;
    HopArgs b = a;
    b.in = static_cast<const char *>(a.in) + (size_t)r * a.rhs_bytes;
    cx<float> A[1][12], B[1][12];
    // past the end the second lane repeats site a and is not stored
    hop_accumulate_pair<P, DAG>(b, ia, has_b ? ib : ia, A, B);
    epi.template operator()<P, 1>(a, ia, true, r, A);
    if (has_b) epi.template operator()<P, 1>(a, ib, true, r, B);
}

template <int P, bool DAG, int MINB>
void launch_k_hop_pair(HopArgs a, const EpiStore &e, cudaStream_t s)
{
    a.ngroups = a.nrhs;
    const int nsb = (a.g.Vh + 2 * kPairThreads - 1) / (2 * kPairThreads);
    k_hop_pair<P, DAG, MINB><<<nsb * a.nrhs, kPairThreads, 0, s>>>(a, e);
}

int sm_count();

template <int P, bool DAG, int NB, int MINB>
void launch_k_hop_gs(HopArgs a, const EpiStore &e, cudaStream_t s)
{
    a.ngroups = (a.nrhs + NB - 1) / NB;
    k_hop_gs<P, DAG, NB, MINB><<<MINB * sm_count(), 128, 0, s>>>(a, e);
}

template <int P, bool DAG, int KIND>
__device__ __forceinline__ void hop_reduce_body(const HopArgs &a, const EpiReduce<KIND> &e)
{
    using R = typename PrecTraits<P>::R;
    constexpr int NV = EpiReduce<KIND>::NV;
    const int r = blockIdx.x % a.nrhs;
    const int sb = blockIdx.x / a.nrhs;
    BiState &st = e.st[r];
    if (__ldcg(&st.done)) return;   // uniform over every block of this rhs
    const int i = sb * blockDim.x + threadIdx.x;
    const bool active = i < a.g.Vh;
    const double coef = e.coef_dev ? __ldcg(e.coef_dev) : e.coef;
    using RedT = typename RedType<R>::T;
    RedT red[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) red[k] = RedT(0);
    if (active) {
        cx<R> acc[1][12];
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[0][k] = acc_zero<R>();
        if constexpr (P == WL_DF) {
            // double-float: the rolled transporter loop (the unrolled one
            // overflows the instruction cache)
            HopArgs b = a;
            b.in = static_cast<const char *>(a.in) + (size_t)r * a.rhs_bytes;
            hop_accumulate_rolled<P, DAG>(b, i, acc[0]);
        } else {
            hop_accumulate<P, DAG, 1>(a, i, r, acc);
        }
        const size_t off = (size_t)r * e.rhs_bytes;
        cx<R> xv[12], o[12];
        SpinorIO<P>::load(static_cast<const char *>(e.xin) + off, a.g.stride, i, xv);
#pragma unroll
        for (int k = 0; k < 12; ++k) o[k] = R(e.a1) * xv[k] + R(coef) * acc[0][k];
        // Reductions use the stored (rounded) values so that they describe
        // exactly the vector the next kernels read.
        SpinorIO<P>::store_rounded(static_cast<char *>(e.out) + off, a.g.stride, i, o);
        if constexpr (KIND == 0) {
            cx<R> rh[12];
            SpinorIO<P>::load(static_cast<const char *>(e.rhat) + off, a.g.stride, i, rh);
            cx<R> d = {R(0), R(0)};
            R n = R(0);
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                d = conjmad(rh[k], o[k], d);
                n = fma(o[k].re, o[k].re, fma(o[k].im, o[k].im, n));
            }
            red[0] = red_cast<RedT>(d.re);
            red[1] = red_cast<RedT>(d.im);
            red[2] = red_cast<RedT>(n);
        } else if constexpr (KIND == 1) {
            cx<R> d = {R(0), R(0)};
            R n = R(0);
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                d = conjmad(o[k], xv[k], d);
                n = fma(o[k].re, o[k].re, fma(o[k].im, o[k].im, n));
            }
            red[0] = red_cast<RedT>(d.re);
            red[1] = red_cast<RedT>(d.im);
            red[2] = red_cast<RedT>(n);
        } else {
            R n = R(0);
#pragma unroll
            for (int k = 0; k < 12; ++k) n = fma(o[k].re, o[k].re, fma(o[k].im, o[k].im, n));
            red[2] = red_cast<RedT>(n);
        }
    }
    double tot[NV];
    if (grid_sum<NV>(red, e.partials + (size_t)r * e.blk_total * kRedNV, &st.ticket[KIND], e.blk_off + sb,
                     e.blk_total, tot) &&
        threadIdx.x == 0) {
        if constexpr (KIND == 0) {
            const double dr = tot[0], di = tot[1];
            const double den = dr * dr + di * di;
            if (!(den > st.brk2 * st.rhat2 * tot[2]) || !isfinite(den)) {
                st.breakdown = 1;
                st.done = 1;
            } else {  // alpha = rho / <rhat, v>
                st.alpha_re = (st.rho_re * dr + st.rho_im * di) / den;
                st.alpha_im = (st.rho_im * dr - st.rho_re * di) / den;
            }
        } else if constexpr (KIND == 1) {
            const double tt = tot[2];
            if (tt > 0.0 && isfinite(tt)) {
                st.omega_re = tot[0] / tt;
                st.omega_im = tot[1] / tt;
            } else {
                st.omega_re = 0.0;
                st.omega_im = 0.0;
            }
        } else if constexpr (KIND == 2) {
            // CG on the normal equations: w = M p, alpha = ||z||^2 / ||w||^2
            const double ww = tot[2];
            if (!(ww > 0.0) || !isfinite(ww)) {
                st.breakdown = 1;
                st.done = 1;
            } else {
                st.alpha_re = st.rho_re / ww;
                st.alpha_im = 0.0;
            }
        } else {
            // z = M^dag r, beta = ||z||^2 / ||z_old||^2 (0 on the first z
            // after a restart), rho = ||z||^2
            const double zz = tot[2];
            if (!isfinite(zz)) {
                st.breakdown = 1;
                st.done = 1;
            } else {
                st.beta_re = (st.iters == 0 || !(st.rho_re > 0.0)) ? 0.0 : zz / st.rho_re;
                st.beta_im = 0.0;
                st.omega_re = st.omega_im = 0.0;
                st.rho_re = zz;
                st.rho_im = 0.0;
            }
        }
    }
}

// Resident blocks per SM the reduction-fused hop asks the register
// allocator for: six (80 registers, no spills) for FP16 storage, where
// occupancy hides the load latency; the other precisions need more
// registers than that (FP32 would spill at 80).
template <int P> struct ReduceMinBlocks {
    static constexpr int value = P == WL_F16 ? 6 : 1;
};

template <int P, bool DAG, int KIND>
__global__ void __launch_bounds__(128, ReduceMinBlocks<P>::value) k_hop_reduce(HopArgs a, EpiReduce<KIND> e)
{
    hop_reduce_body<P, DAG, KIND>(a, e);
}

// ------------------------------------------------------------ launchers
// Instantiated per precision in hop_<prec>.cu.

template <int P, bool DAG, int NB, int MINB>
void launch_k_hop(HopArgs a, const EpiStore &e, cudaStream_t s)
{
    a.ngroups = (a.nrhs + NB - 1) / NB;
    const int nsb = (a.g.Vh + 127) / 128;
    k_hop<P, DAG, NB, MINB><<<nsb * a.ngroups, 128, 0, s>>>(a, e);
}

template <int P, bool DAG, int MINB>
void launch_k_hop_rolled(HopArgs a, const EpiStore &e, cudaStream_t s)
{
    a.ngroups = a.nrhs;
    const int nsb = (a.g.Vh + 127) / 128;
    k_hop_rolled<P, DAG, MINB><<<nsb * a.nrhs, 128, 0, s>>>(a, e);
}

template <int P, bool DAG, int KIND>
void launch_k_hop_reduce(const HopArgs &a, const EpiReduce<KIND> &e, cudaStream_t s)
{
    const int nsb = (a.g.Vh + 127) / 128;
    k_hop_reduce<P, DAG, KIND><<<nsb * a.nrhs, 128, 0, s>>>(a, e);
}

template <int P, int KIND>
void launch_reduce_kind(int dagger, const HopArgs &a, const void *epi, cudaStream_t s)
{
    const auto &e = *static_cast<const EpiReduce<KIND> *>(epi);
    if (dagger)
        launch_k_hop_reduce<P, true, KIND>(a, e, s);
    else
        launch_k_hop_reduce<P, false, KIND>(a, e, s);
}

// Returned by a launcher whose variant does not apply to the lattice.
constexpr int WL_VARIANT_NA = -100;

// TMA-staged hop (hop_tma.cu), FP32 and FP16, variants 9000 + rhs per tile.
int hop_launch_tma(int prec, int variant, int dagger, const HopArgs &a, const EpiStore &e, cudaStream_t s);

// Per-precision entry points (hop_<prec>.cu).  variant: see hop_variants().
template <int P> int hop_launch_prec(int variant, int dagger, const HopArgs &a, const EpiStore &e, cudaStream_t s);
template <int P> int hop_reduce_launch_prec(int kind, int dagger, const HopArgs &a, const void *epi, cudaStream_t s);

}  // namespace wl
