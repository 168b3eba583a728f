// Host dispatch of the hop kernels and the dslash entry points of the C ABI.
#include "hop.cuh"

namespace wl {

// ------------------------------------------------------------------ launch

static const void *links_of(wl_gauge *g, int prec, int parity) { return g->links[prec_index(prec)][parity]; }

// SM count of the current device (grid-stride launches).
int sm_count()
{
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
        v > 0)
        return v;
    return 1;
}

static int check_links(wl_gauge *g, int prec)
{
    if (!(g->prec_mask & prec) || !links_of(g, prec, 0)) {
        set_error("gauge handle holds no links of the requested precision");
        return WL_ERR_ARG;
    }
    return WL_OK;
}

int hop_ex(wl_gauge *g, const Vec &in, const Vec &out, const Vec *x1, double a1, const Vec *x2, double a2,
           double coef, int out_parity, int dagger, int rhs_block, const int *skip, int skip_stride, cudaStream_t s,
           const Vec *out_raw)
{
    WL_TRY(check_links(g, in.prec));
    if (in.prec != out.prec || (x1 && x1->prec != in.prec) || (x2 && x2->prec != in.prec)) {
        set_error("hop: precision mismatch");
        return WL_ERR_ARG;
    }
    HopArgs a;
    a.g = g->lat->geom;
    a.out_parity = out_parity;
    a.nrhs = in.nrhs;
    a.ngroups = in.nrhs;
    a.in = in.ptr;
    a.rhs_bytes = in.rhs_bytes;
    a.links_out = links_of(g, in.prec, out_parity);
    a.links_in = links_of(g, in.prec, 1 - out_parity);
    a.skip = skip;
    a.skip_stride = skip_stride;
    EpiStore e;
    e.out = out.ptr;
    e.out_raw = out_raw ? out_raw->ptr : nullptr;
    e.x1 = x1 ? x1->ptr : nullptr;
    e.x2 = x2 ? x2->ptr : nullptr;
    e.a1 = a1;
    e.a2 = a2;
    e.coef = coef;
    e.rhs_bytes = out.rhs_bytes;
    if (out.rhs_bytes != in.rhs_bytes) { set_error("hop: rhs stride mismatch"); return WL_ERR_ARG; }
    const int variant = hop_variant_for(g, in.prec, in.nrhs, rhs_block);
    int st = WL_ERR_ARG;
    switch (in.prec) {
    case WL_F64: st = hop_launch_prec<WL_F64>(variant, dagger, a, e, s); break;
    case WL_F32: st = hop_launch_prec<WL_F32>(variant, dagger, a, e, s); break;
    case WL_F16: st = hop_launch_prec<WL_F16>(variant, dagger, a, e, s); break;
    case WL_DF: st = hop_launch_prec<WL_DF>(variant, dagger, a, e, s); break;
    default: set_error("hop: bad precision"); return WL_ERR_ARG;
    }
    if (st == WL_VARIANT_NA) return WL_ERR_ARG;
    WL_TRY(st);
    WL_CUDA_TRY(cudaGetLastError());
    note_launch(s);
    return WL_OK;
}

int hop(wl_gauge *g, const Vec &in, const Vec &out, const Vec *x, double coef, int out_parity, int dagger,
        int rhs_block, cudaStream_t s)
{
    return hop_ex(g, in, out, x, 1.0, nullptr, 0.0, coef, out_parity, dagger, rhs_block, nullptr, 0, s);
}

template <int KIND>
static int hop_reduce_k(wl_gauge *g, const Vec &tmp, const Vec &xin, double a1, const Vec &out, const Vec &rhat,
                        double coef, const double *coef_dev, int out_parity, int dagger, BiState *state,
                        double *partials, int blk_off, int blk_total, cudaStream_t s)
{
    WL_TRY(check_links(g, tmp.prec));
    HopArgs a;
    a.g = g->lat->geom;
    a.out_parity = out_parity;
    a.nrhs = tmp.nrhs;
    a.ngroups = tmp.nrhs;
    a.in = tmp.ptr;
    a.rhs_bytes = tmp.rhs_bytes;
    a.links_out = links_of(g, tmp.prec, out_parity);
    a.links_in = links_of(g, tmp.prec, 1 - out_parity);
    a.skip = &state[0].done;
    a.skip_stride = sizeof(BiState) / sizeof(int);
    EpiReduce<KIND> e;
    e.out = out.ptr;
    e.xin = xin.ptr;
    e.rhat = rhat.ptr;
    e.a1 = a1;
    e.coef = coef;
    e.coef_dev = coef_dev;
    e.blk_off = blk_off;
    e.blk_total = blk_total;
    e.rhs_bytes = out.rhs_bytes;
    e.st = state;
    e.partials = partials;
    int st = WL_ERR_ARG;
    switch (tmp.prec) {
    case WL_F64: st = hop_reduce_launch_prec<WL_F64>(KIND, dagger, a, &e, s); break;
    case WL_F32: st = hop_reduce_launch_prec<WL_F32>(KIND, dagger, a, &e, s); break;
    case WL_F16: st = hop_reduce_launch_prec<WL_F16>(KIND, dagger, a, &e, s); break;
    case WL_DF: st = hop_reduce_launch_prec<WL_DF>(KIND, dagger, a, &e, s); break;
    default: set_error("hop_reduce: bad precision"); return WL_ERR_ARG;
    }
    WL_TRY(st);
    WL_CUDA_TRY(cudaGetLastError());
    note_launch(s);
    return WL_OK;
}

int hop_reduce(wl_gauge *g, int kind, const Vec &tmp, const Vec &xin, double a1, const Vec &out, const Vec &rhat,
               double coef, const double *coef_dev, int out_parity, int dagger, BiState *state, double *partials,
               int blk_off, int blk_total, cudaStream_t s)
{
    switch (kind) {
    case 0: return hop_reduce_k<0>(g, tmp, xin, a1, out, rhat, coef, coef_dev, out_parity, dagger, state, partials,
                                   blk_off, blk_total, s);
    case 1: return hop_reduce_k<1>(g, tmp, xin, a1, out, rhat, coef, coef_dev, out_parity, dagger, state, partials,
                                   blk_off, blk_total, s);
    case 2: return hop_reduce_k<2>(g, tmp, xin, a1, out, rhat, coef, coef_dev, out_parity, dagger, state, partials,
                                   blk_off, blk_total, s);
    case 3: return hop_reduce_k<3>(g, tmp, xin, a1, out, rhat, coef, coef_dev, out_parity, dagger, state, partials,
                                   blk_off, blk_total, s);
    default: set_error("hop_reduce: bad kind"); return WL_ERR_ARG;
    }
}

}  // namespace wl

using namespace wl;

// ---------------------------------------------------------------- C ABI

// In the bounds-checked build the dslash calls synchronise the stream and
// report a recorded out-of-range index.
static int dslash_checked(int st, void *stream)
{
#ifdef WL_CHECKED
    if (st == WL_OK) WL_CUDA_TRY(cudaStreamSynchronize(as_stream(stream)));
    return checked_result(st);
#else
    (void)stream;
    return st;
#endif
}

extern "C" int wilson_hop(wl_gauge *g, const void *in, void *out, const void *x, double coef, int prec,
                          int out_parity, int dagger, void *stream)
{
    if (!g || !in || !out || !valid_prec(prec) || (out_parity != 0 && out_parity != 1) || in == out) {
        set_error("wilson_hop: bad argument");
        return WL_ERR_ARG;
    }
    Vec vi, vo, vx;
    vi.ptr = const_cast<void *>(in);
    vi.prec = vo.prec = vx.prec = prec;
    vi.rhs_bytes = vo.rhs_bytes = vx.rhs_bytes = spinor_bytes(g->lat->geom, prec);
    vo.ptr = out;
    vx.ptr = const_cast<void *>(x);
    return dslash_checked(hop(g, vi, vo, x ? &vx : nullptr, coef, out_parity, dagger ? 1 : 0, 1, as_stream(stream)),
                          stream);
}

extern "C" int wilson_hop_multi(wl_gauge *g, const void *in, void *out, const void *x, double coef, int prec,
                                int out_parity, int dagger, int n_rhs, size_t rhs_stride, int rhs_block,
                                void *stream)
{
    bool known_variant = rhs_block >= 0;
    if (rhs_block < 0 && valid_prec(prec))
        for (int v : hop_variants(prec)) known_variant |= (v == -rhs_block);
    if (!g || !in || !out || !valid_prec(prec) || (out_parity != 0 && out_parity != 1) || in == out || n_rhs < 1 ||
        !known_variant || rhs_block > 4 || rhs_block == 3 || (rhs_stride & 255) ||
        rhs_stride < spinor_bytes(g->lat->geom, prec)) {
        set_error("wilson_hop_multi: bad argument");
        return WL_ERR_ARG;
    }
    Vec vi, vo, vx;
    vi.ptr = const_cast<void *>(in);
    vo.ptr = out;
    vx.ptr = const_cast<void *>(x);
    vi.prec = vo.prec = vx.prec = prec;
    vi.nrhs = vo.nrhs = vx.nrhs = n_rhs;
    vi.rhs_bytes = vo.rhs_bytes = vx.rhs_bytes = rhs_stride;
    return dslash_checked(hop(g, vi, vo, x ? &vx : nullptr, coef, out_parity, dagger ? 1 : 0, rhs_block,
                              as_stream(stream)), stream);
}

static int dslash_common(wl_gauge *g, const void *in, void *out, double kappa, int prec, int op, int dagger,
                         void *stream)
{
    if (!g || !in || !out || in == out || !valid_prec(prec) || op < WL_OP_HOP || op > WL_OP_MPREC) {
        set_error("wilson_dslash: bad argument");
        return WL_ERR_ARG;
    }
    WL_TRY(check_links(g, prec));
    std::lock_guard<std::mutex> lock(g->mu);
    cudaStream_t s = as_stream(stream);
    const Geom &geo = g->lat->geom;
    Vec ie, io, oe, oo;
    WL_TRY(make_vec(g, "dslash_ie", prec, 1, &ie));
    WL_TRY(make_vec(g, "dslash_io", prec, 1, &io));
    WL_TRY(make_vec(g, "dslash_oe", prec, 1, &oe));
    WL_TRY(make_vec(g, "dslash_oo", prec, 1, &oo));
    const void *cin[1] = {in};
    void *cout[1] = {out};
    WL_TRY(import_full(geo, cin, ie, io, s));
    if (op == WL_OP_HOP) {
        WL_TRY(hop(g, io, oe, nullptr, 1.0, WL_EVEN, dagger, 1, s));
        WL_TRY(hop(g, ie, oo, nullptr, 1.0, WL_ODD, dagger, 1, s));
    } else if (op == WL_OP_M) {
        WL_TRY(hop(g, io, oe, &ie, -kappa, WL_EVEN, dagger, 1, s));
        WL_TRY(hop(g, ie, oo, &io, -kappa, WL_ODD, dagger, 1, s));
    } else {
        // out_e = in_e - kappa^2 D_eo D_oe in_e.  With dagger hops this is
        // 1 - kappa^2 g5 D_eo D_oe g5 = M_prec^dag.
        WL_TRY(hop(g, ie, oo, nullptr, 1.0, WL_ODD, dagger, 1, s));
        WL_TRY(hop(g, oo, oe, &ie, -kappa * kappa, WL_EVEN, dagger, 1, s));
        WL_CUDA_TRY(cudaMemsetAsync(oo.ptr, 0, spinor_bytes(geo, prec), s));
    }
    WL_TRY(export_full(geo, oe, oo, cout, s));
    return WL_OK;
}

extern "C" int wilson_dslash(wl_gauge *g, const void *in, void *out, double kappa, int prec, int op, void *stream)
{
    return dslash_checked(dslash_common(g, in, out, kappa, prec, op, 0, stream), stream);
}

extern "C" int wilson_dslash_dag(wl_gauge *g, const void *in, void *out, double kappa, int prec, int op,
                                 void *stream)
{
    return dslash_checked(dslash_common(g, in, out, kappa, prec, op, 1, stream), stream);
}
