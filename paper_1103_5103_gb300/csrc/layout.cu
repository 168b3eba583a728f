// Geometry, handles, workspace and the canonical <-> internal layout kernels
// (Section 4, Eqs. 7-8: structure-of-arrays fields, even sites first).
#include <atomic>
#include <cstdio>
#include <cstring>
#include <string>

#include <mutex>
#include <vector>

#include "internal.h"

namespace wl {

static thread_local std::string g_last_error;
static std::atomic<long long> g_launches{0};

void set_error(const std::string &msg) { g_last_error = msg; }

void note_launch(cudaStream_t s)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive) return;
    g_launches.fetch_add(1, std::memory_order_relaxed);
}

void add_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

size_t spinor_bytes(const Geom &g, int prec) { return (size_t)spinor_site_bytes(prec) * g.stride; }

// Readers of the per-translation-unit violation words of the bounds-checked
// build (each unit registers one at static initialisation).
static std::vector<int (*)(unsigned long long *, bool)> &checked_readers()
{
    static std::vector<int (*)(unsigned long long *, bool)> v;
    return v;
}
static std::mutex g_checked_mu;

int checked_register(int (*reader)(unsigned long long *, bool))
{
    std::lock_guard<std::mutex> lock(g_checked_mu);
    checked_readers().push_back(reader);
    return 1;
}

int checked_status(unsigned long long *first, bool reset)
{
    *first = 0;
    std::lock_guard<std::mutex> lock(g_checked_mu);
    for (auto rd : checked_readers()) {
        unsigned long long v = 0;
        WL_TRY(rd(&v, reset));
        if (v && !*first) *first = v;
    }
    return WL_OK;
}

int HostPinned::get(const std::string &name, size_t bytes, void **out)
{
    DevBuf &b = bufs[name];
    if (b.bytes < bytes) {
        if (b.ptr) cudaFreeHost(b.ptr);
        b.ptr = nullptr;
        b.bytes = 0;
        cudaError_t e = cudaMallocHost(&b.ptr, bytes);
        if (e != cudaSuccess) {
            b.ptr = nullptr;
            set_error("pinned staging '" + name + "': " + cudaGetErrorString(e));
            return WL_ERR_OOM;
        }
        b.bytes = bytes;
    }
    *out = b.ptr;
    return WL_OK;
}

void HostPinned::release()
{
    for (auto &kv : bufs)
        if (kv.second.ptr) cudaFreeHost(kv.second.ptr);
    bufs.clear();
}

int Workspace::get(const std::string &name, size_t bytes, void **out)
{
    DevBuf &b = bufs[name];
    if (b.bytes < bytes) {
        if (b.ptr) cudaFree(b.ptr);
        b.ptr = nullptr;
        b.bytes = 0;
        cudaError_t e = cudaMalloc(&b.ptr, bytes);
        if (e != cudaSuccess) {
            set_error("workspace '" + name + "' cudaMalloc(" + std::to_string(bytes) + "): " + cudaGetErrorString(e));
            b.ptr = nullptr;
            return e == cudaErrorMemoryAllocation ? WL_ERR_OOM : WL_ERR_CUDA;
        }
        b.bytes = bytes;
    }
    *out = b.ptr;
    return WL_OK;
}

void Workspace::release()
{
    for (auto &kv : bufs)
        if (kv.second.ptr) cudaFree(kv.second.ptr);
    bufs.clear();
}

int make_vec(wl_gauge *g, const std::string &name, int prec, int nrhs, Vec *v)
{
    v->prec = prec;
    v->nrhs = nrhs;
    v->rhs_bytes = (spinor_bytes(g->lat->geom, prec) + 255) & ~(size_t)255;
    return g->ws.get(name, v->rhs_bytes * nrhs, &v->ptr);
}

// ------------------------------------------------------------ layout kernels

template <int P>
__global__ void k_import(Geom g, const double2 *__restrict__ canon, void *out, int parity)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.Vh) return;
    const Coord c = site_coord(g, i, parity);
    const size_t lex = c.x + (size_t)g.X * (c.y + (size_t)g.Y * (c.z + (size_t)g.Z * c.t));
    using R = typename PrecTraits<P>::R;
    cx<R> v[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        double2 t = canon[lex * 12 + k];
        v[k] = {Conv<R>::from(t.x), Conv<R>::from(t.y)};
    }
    SpinorIO<P>::store(out, g.stride, i, v);
}

template <int P>
__global__ void k_export(Geom g, const void *in, double2 *__restrict__ canon, int parity)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.Vh) return;
    const Coord c = site_coord(g, i, parity);
    const size_t lex = c.x + (size_t)g.X * (c.y + (size_t)g.Y * (c.z + (size_t)g.Z * c.t));
    using R = typename PrecTraits<P>::R;
    cx<R> v[12];
    SpinorIO<P>::load(in, g.stride, i, v);
#pragma unroll
    for (int k = 0; k < 12; ++k) canon[lex * 12 + k] = make_double2(to_double(v[k].re), to_double(v[k].im));
}

// Both parities at once, through shared memory, so that the canonical side
// is read or written in whole lines: a block takes the 128 consecutive
// lexicographic sites 128 b .. 128 b + 127, i.e. even-odd indices 64 b ..
// 64 b + 63 of both parities (eo index = floor(lex / 2)).  The staging
// buffer is component-major with a stride of 129 (no bank conflicts).
constexpr int kFullSites = 128;

__device__ __forceinline__ int lex_parity(const Geom &g, size_t n)
{
    const int x = (int)(n % g.X);
    size_t r = n / g.X;
    const int y = (int)(r % g.Y);
    r /= g.Y;
    const int z = (int)(r % g.Z);
    const int t = (int)(r / g.Z);
    return (x + y + z + t) & 1;
}

template <int P>
__global__ void __launch_bounds__(kFullSites) k_export_full(Geom g, const void *even, const void *odd,
                                                            double2 *__restrict__ canon)
{
    __shared__ double2 sm[12 * (kFullSites + 1)];
    const size_t V = (size_t)g.Vh * 2;
    const size_t ntiles = (V + kFullSites - 1) / kFullSites;
    // tiles strided by the grid: a reduced grid (the overlapped export of
    // the multi-mass solver) occupies a few SMs while other work runs
    for (size_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const size_t n0 = tile * kFullSites;
        const size_t n = n0 + threadIdx.x;
        if (n < V) {
            using R = typename PrecTraits<P>::R;
            cx<R> v[12];
            SpinorIO<P>::load(lex_parity(g, n) ? odd : even, g.stride, (int)(n >> 1), v);
#pragma unroll
            for (int k = 0; k < 12; ++k)
                sm[k * (kFullSites + 1) + threadIdx.x] = make_double2(to_double(v[k].re), to_double(v[k].im));
        }
        __syncthreads();
        const size_t e0 = n0 * 12, e_end = V * 12;
#pragma unroll
        for (int j = 0; j < 12; ++j) {
            const int e = j * kFullSites + threadIdx.x;
            if (e0 + e < e_end) canon[e0 + e] = sm[(e % 12) * (kFullSites + 1) + e / 12];
        }
        __syncthreads();   // sm is refilled by the next tile
    }
}

template <int P>
__global__ void __launch_bounds__(kFullSites) k_import_full(Geom g, const double2 *__restrict__ canon, void *even,
                                                            void *odd)
{
    __shared__ double2 sm[12 * (kFullSites + 1)];
    const size_t V = (size_t)g.Vh * 2;
    const size_t n0 = (size_t)blockIdx.x * kFullSites;
    const size_t e0 = n0 * 12, e_end = V * 12;
#pragma unroll
    for (int j = 0; j < 12; ++j) {
        const int e = j * kFullSites + threadIdx.x;
        if (e0 + e < e_end) sm[(e % 12) * (kFullSites + 1) + e / 12] = canon[e0 + e];
    }
    __syncthreads();
    const size_t n = n0 + threadIdx.x;
    if (n < V) {
        using R = typename PrecTraits<P>::R;
        cx<R> v[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const double2 t = sm[k * (kFullSites + 1) + threadIdx.x];
            v[k] = {Conv<R>::from(t.x), Conv<R>::from(t.y)};
        }
        SpinorIO<P>::store(lex_parity(g, n) ? odd : even, g.stride, (int)(n >> 1), v);
    }
}

// Pack U_mu at the sites of one parity: rows 0 and 1 for F32, all three
// rows for F64 and F16 (as given) and DF (row 2 formed in FP64).
template <int P>
__global__ void k_pack_links(Geom g, const double2 *__restrict__ U, void *out, int parity)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int mu = blockIdx.y;
    if (i >= g.Vh) return;
    const Coord c = site_coord(g, i, parity);
    const size_t V = (size_t)g.Vh * 2;
    const size_t lex = c.x + (size_t)g.X * (c.y + (size_t)g.Y * (c.z + (size_t)g.Z * c.t));
    const double2 *u = U + ((size_t)mu * V + lex) * 9;
    char *dir = static_cast<char *>(out) + (size_t)mu * link_dir_bytes(P, g.stride);
    if (P == WL_F64) {
        double2 *p = reinterpret_cast<double2 *>(dir);
        for (int k = 0; k < 9; ++k) p[(size_t)k * g.stride + i] = u[k];
    } else if (P == WL_F32) {
        float4 *p = reinterpret_cast<float4 *>(dir);
        for (int k = 0; k < 3; ++k) {
            double2 a = u[2 * k], b = u[2 * k + 1];
            p[(size_t)k * g.stride + i] = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
        }
    } else if (P == WL_DF) {
        // rows 0, 1 as given; row 2 = conj(row 0 x row 1) in FP64, the same
        // relation the other precisions rebuild on the fly
        double2 w[9];
        for (int k = 0; k < 6; ++k) w[k] = u[k];
        for (int c = 0; c < 3; ++c) {
            const double2 a1 = w[(c + 1) % 3], a2 = w[(c + 2) % 3], b1 = w[3 + (c + 1) % 3], b2 = w[3 + (c + 2) % 3];
            const double re = (a1.x * b2.x - a1.y * b2.y) - (a2.x * b1.x - a2.y * b1.y);
            const double im = (a1.x * b2.y + a1.y * b2.x) - (a2.x * b1.y + a2.y * b1.x);
            w[6 + c] = make_double2(re, -im);
        }
        float4 *p = reinterpret_cast<float4 *>(dir);
        for (int k = 0; k < 9; ++k) {
            const df re(w[k].x), im(w[k].y);
            p[(size_t)k * g.stride + i] = make_float4(re.hi, re.lo, im.hi, im.lo);
        }
    } else {
        uint2 *p = reinterpret_cast<uint2 *>(dir);
        for (int k = 0; k < 4; ++k) {
            double2 a = u[2 * k], b = u[2 * k + 1];
            uint2 t;
            t.x = pack_half2((float)a.x, (float)a.y);
            t.y = pack_half2((float)b.x, (float)b.y);
            p[(size_t)k * g.stride + i] = t;
        }
        reinterpret_cast<unsigned *>(p + (size_t)4 * g.stride)[i] = pack_half2((float)u[8].x, (float)u[8].y);
    }
}

template <int P>
static int launch_import(const Geom &g, const void *canon, void *out, int parity, cudaStream_t s)
{
    const int th = 128, bl = (g.Vh + th - 1) / th;
    k_import<P><<<bl, th, 0, s>>>(g, static_cast<const double2 *>(canon), out, parity);
    WL_CUDA_TRY(cudaGetLastError());
    note_launch(s);
    return WL_OK;
}

template <int P>
static int launch_export(const Geom &g, const void *in, void *canon, int parity, cudaStream_t s)
{
    const int th = 128, bl = (g.Vh + th - 1) / th;
    k_export<P><<<bl, th, 0, s>>>(g, in, static_cast<double2 *>(canon), parity);
    WL_CUDA_TRY(cudaGetLastError());
    note_launch(s);
    return WL_OK;
}

template <int P>
static int launch_full(const Geom &g, const void *canon_in, void *canon_out, const void *even_in, const void *odd_in,
                       void *even_out, void *odd_out, cudaStream_t s, int max_blocks = 0)
{
    unsigned bl = (unsigned)(((size_t)g.Vh * 2 + kFullSites - 1) / kFullSites);
    if (max_blocks > 0 && canon_out && bl > (unsigned)max_blocks) bl = (unsigned)max_blocks;
    if (canon_out)
        k_export_full<P><<<bl, kFullSites, 0, s>>>(g, even_in, odd_in, static_cast<double2 *>(canon_out));
    else
        k_import_full<P><<<bl, kFullSites, 0, s>>>(g, static_cast<const double2 *>(canon_in), even_out, odd_out);
    WL_CUDA_TRY(cudaGetLastError());
    note_launch(s);
    return WL_OK;
}

int export_full(const Geom &g, const Vec &even, const Vec &odd, void *const *canon, cudaStream_t s, int max_blocks)
{
    if (even.prec != odd.prec || even.nrhs != odd.nrhs) { set_error("export_full: parity mismatch"); return WL_ERR_ARG; }
    for (int r = 0; r < even.nrhs; ++r) {
        const void *e = even.rhs(r), *o = odd.rhs(r);
        const int mb = max_blocks;
        int st = even.prec == WL_F64   ? launch_full<WL_F64>(g, nullptr, canon[r], e, o, nullptr, nullptr, s, mb)
                 : even.prec == WL_F32 ? launch_full<WL_F32>(g, nullptr, canon[r], e, o, nullptr, nullptr, s, mb)
                 : even.prec == WL_DF  ? launch_full<WL_DF>(g, nullptr, canon[r], e, o, nullptr, nullptr, s, mb)
                                       : launch_full<WL_F16>(g, nullptr, canon[r], e, o, nullptr, nullptr, s, mb);
        WL_TRY(st);
    }
    return WL_OK;
}

int import_full(const Geom &g, const void *const *canon, const Vec &even, const Vec &odd, cudaStream_t s)
{
    if (even.prec != odd.prec || even.nrhs != odd.nrhs) { set_error("import_full: parity mismatch"); return WL_ERR_ARG; }
    for (int r = 0; r < even.nrhs; ++r) {
        void *e = even.rhs(r), *o = odd.rhs(r);
        int st = even.prec == WL_F64   ? launch_full<WL_F64>(g, canon[r], nullptr, nullptr, nullptr, e, o, s)
                 : even.prec == WL_F32 ? launch_full<WL_F32>(g, canon[r], nullptr, nullptr, nullptr, e, o, s)
                 : even.prec == WL_DF  ? launch_full<WL_DF>(g, canon[r], nullptr, nullptr, nullptr, e, o, s)
                                       : launch_full<WL_F16>(g, canon[r], nullptr, nullptr, nullptr, e, o, s);
        WL_TRY(st);
    }
    return WL_OK;
}

int import_spinors(const Geom &g, const void *const *canon, const Vec &out, int parity, cudaStream_t s)
{
    for (int r = 0; r < out.nrhs; ++r) {
        int st = out.prec == WL_F64   ? launch_import<WL_F64>(g, canon[r], out.rhs(r), parity, s)
                 : out.prec == WL_F32 ? launch_import<WL_F32>(g, canon[r], out.rhs(r), parity, s)
                 : out.prec == WL_DF  ? launch_import<WL_DF>(g, canon[r], out.rhs(r), parity, s)
                                      : launch_import<WL_F16>(g, canon[r], out.rhs(r), parity, s);
        WL_TRY(st);
    }
    return WL_OK;
}

int export_spinors(const Geom &g, const Vec &in, void *const *canon, int parity, cudaStream_t s)
{
    for (int r = 0; r < in.nrhs; ++r) {
        int st = in.prec == WL_F64   ? launch_export<WL_F64>(g, in.rhs(r), canon[r], parity, s)
                 : in.prec == WL_F32 ? launch_export<WL_F32>(g, in.rhs(r), canon[r], parity, s)
                 : in.prec == WL_DF  ? launch_export<WL_DF>(g, in.rhs(r), canon[r], parity, s)
                                     : launch_export<WL_F16>(g, in.rhs(r), canon[r], parity, s);
        WL_TRY(st);
    }
    return WL_OK;
}

}  // namespace wl

using namespace wl;

// ---------------------------------------------------------------- C ABI

extern "C" const char *wl_last_error(void) { return g_last_error.c_str(); }

extern "C" int wl_launch_count(long long *out)
{
    if (!out) { set_error("wl_launch_count: NULL"); return WL_ERR_ARG; }
    *out = g_launches.load();
    return WL_OK;
}

extern "C" int wl_is_checked_build(void)
{
#ifdef WL_CHECKED
    return 1;
#else
    return 0;
#endif
}

extern "C" int wl_checked_status(unsigned long long *first, int reset)
{
    if (!first) {
        set_error("wl_checked_status: NULL");
        return WL_ERR_ARG;
    }
    WL_CUDA_TRY(cudaDeviceSynchronize());
    return checked_status(first, reset != 0);
}

extern "C" int wl_params_default(wl_solver_params *p)
{
    if (!p) { set_error("wl_params_default: NULL"); return WL_ERR_ARG; }
    p->tol = 1e-10;
    p->max_iter = 100000;
    p->inner_prec = WL_F32;
    p->inner_tol = 0.0;
    p->max_restarts = 100;
    p->guess = WL_GUESS_POLY;
    p->mode = WL_MODE_GRAPH;
    p->rhs_block = 0;
    p->graph_iters = 8;
    p->eo = 1;
    p->outer_prec = WL_F64;
    p->shadow = nullptr;
    p->guess_max = 0;
    p->reliable = 0;
    p->inner_solver = WL_SOLVER_BICGSTAB;
    p->verify_full = 0;
    p->outer_blocks_per_sm = 0;
    p->inner_refine = 0;
    return WL_OK;
}

extern "C" int wl_lattice_create(const int dims[4], int antiperiodic_t, wl_lattice **out)
{
    if (!dims || !out) { set_error("wl_lattice_create: NULL argument"); return WL_ERR_ARG; }
    long V = 1;
    for (int k = 0; k < 4; ++k) {
        if (dims[k] < 2 || (dims[k] & 1)) {
            set_error("wl_lattice_create: every extent must be even and >= 2 (got " + std::to_string(dims[k]) + ")");
            return WL_ERR_ARG;
        }
        V *= dims[k];
    }
    if (V >= (1L << 31) / 12) { set_error("wl_lattice_create: volume too large"); return WL_ERR_ARG; }
    wl_lattice *l = new wl_lattice;
    std::memcpy(l->dims, dims, sizeof(int) * 4);
    l->antiperiodic = antiperiodic_t ? 1 : 0;
    l->volume = V;
    Geom &g = l->geom;
    g.X = dims[0]; g.Y = dims[1]; g.Z = dims[2]; g.T = dims[3];
    g.Xh = dims[0] / 2;
    g.Vh = (int)(V / 2);
    g.stride = (g.Vh + 63) & ~63;
    g.antiperiodic = l->antiperiodic;
    *out = l;
    return WL_OK;
}

extern "C" int wl_lattice_destroy(wl_lattice *lat)
{
    delete lat;
    return WL_OK;
}

extern "C" int wl_spinor_bytes(const wl_lattice *lat, int prec, size_t *bytes)
{
    if (!lat || !bytes || !valid_prec(prec)) { set_error("wl_spinor_bytes: bad argument"); return WL_ERR_ARG; }
    *bytes = spinor_bytes(lat->geom, prec);
    return WL_OK;
}

extern "C" int wl_spinor_import(const wl_lattice *lat, const void *canon, void *internal, int prec, int parity,
                                void *stream)
{
    if (!lat || !canon || !internal || !valid_prec(prec) || (parity != 0 && parity != 1)) {
        set_error("wl_spinor_import: bad argument");
        return WL_ERR_ARG;
    }
    Vec v;
    v.ptr = internal;
    v.prec = prec;
    v.nrhs = 1;
    const void *c[1] = {canon};
    return import_spinors(lat->geom, c, v, parity, as_stream(stream));
}

extern "C" int wl_spinor_export(const wl_lattice *lat, const void *internal, void *canon, int prec, int parity,
                                void *stream)
{
    if (!lat || !canon || !internal || !valid_prec(prec) || (parity != 0 && parity != 1)) {
        set_error("wl_spinor_export: bad argument");
        return WL_ERR_ARG;
    }
    Vec v;
    v.ptr = const_cast<void *>(internal);
    v.prec = prec;
    v.nrhs = 1;
    void *c[1] = {canon};
    return export_spinors(lat->geom, v, c, parity, as_stream(stream));
}

// Largest deviation of the canonical links from SU(3): max over links of
// the entries of |U U^dag - 1| and of |det U - 1| (each as max(|re|, |im|)).
// A NaN counts as +inf.  Blocks combine with an atomic max on the bit
// pattern, which orders non-negative doubles (and +inf) like their values.
static __device__ __forceinline__ void dev_max(double &m, double v)
{
    if (!(v <= m)) m = (v != v) ? INFINITY : v;
}

static __global__ void k_su3_deviation(const double2 *__restrict__ U, size_t nlinks, unsigned long long *out)
{
    double m = 0.0;
    for (size_t l = (size_t)blockIdx.x * blockDim.x + threadIdx.x; l < nlinks; l += (size_t)gridDim.x * blockDim.x) {
        cx<double> u[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const double2 t = U[l * 9 + k];
            u[k] = {t.x, t.y};
        }
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = a; b < 3; ++b) {
                cx<double> s = {a == b ? -1.0 : 0.0, 0.0};
#pragma unroll
                for (int c = 0; c < 3; ++c) s = conjmad(u[3 * b + c], u[3 * a + c], s);  // (U U^dag)_ab - delta_ab
                dev_max(m, fabs(s.re));
                dev_max(m, fabs(s.im));
            }
        const cx<double> det = u[0] * (u[4] * u[8] - u[5] * u[7]) - u[1] * (u[3] * u[8] - u[5] * u[6]) +
                               u[2] * (u[3] * u[7] - u[4] * u[6]);
        dev_max(m, fabs(det.re - 1.0));
        dev_max(m, fabs(det.im));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dev_max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// Links further than this from SU(3) are rejected: the 12-real formats
// rebuild the third row as conj(row 0 x row 1), which is the link only for
// SU(3) matrices.
constexpr double kSU3Tol = 1e-6;

static int su3_deviation(const Geom &geo, const void *U, double *dev, cudaStream_t s)
{
    unsigned long long *d = nullptr, h = 0;
    int dev_id = 0, nsm = 0;
    WL_CUDA_TRY(cudaGetDevice(&dev_id));
    WL_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev_id));
    WL_CUDA_TRY(cudaMalloc(&d, sizeof(unsigned long long)));
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) {
        const size_t nlinks = (size_t)4 * geo.Vh * 2;
        const unsigned grid = (unsigned)std::min<size_t>((nlinks + 255) / 256, (size_t)nsm * 8);
        k_su3_deviation<<<grid, 256, 0, s>>>(static_cast<const double2 *>(U), nlinks, d);
        note_launch(s);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d);
    if (e != cudaSuccess) {
        set_error(std::string("wl_gauge_create: ") + cudaGetErrorString(e));
        return WL_ERR_CUDA;
    }
    std::memcpy(dev, &h, sizeof(double));
    return WL_OK;
}

extern "C" int wl_gauge_create(wl_lattice *lat, const void *U, unsigned prec_mask, void *stream, wl_gauge **out)
{
    if (!lat || !U || !out || !(prec_mask & (WL_F64 | WL_F32 | WL_F16 | WL_DF)) || (prec_mask & ~15u)) {
        set_error("wl_gauge_create: bad argument");
        return WL_ERR_ARG;
    }
    cudaStream_t s = as_stream(stream);
    {
        double dev = 0.0;
        WL_TRY(su3_deviation(lat->geom, U, &dev, s));
        if (!(dev <= kSU3Tol)) {
            char msg[160];
            std::snprintf(msg, sizeof(msg), "wl_gauge_create: links are not SU(3) (largest deviation %.3g > %.0e)",
                          dev, kSU3Tol);
            set_error(msg);
            return WL_ERR_ARG;
        }
    }
    wl_gauge *g = new wl_gauge;
    g->lat = lat;
    g->prec_mask = prec_mask;
    std::memset(g->links, 0, sizeof(g->links));
    const Geom &geo = lat->geom;
    const int precs[4] = {WL_F64, WL_F32, WL_F16, WL_DF};
    for (int k = 0; k < 4; ++k) {
        const int P = precs[k];
        const int pi = prec_index(P);
        if (!(prec_mask & P)) continue;
        for (int par = 0; par < 2; ++par) {
            const size_t bytes = 4 * link_dir_bytes(P, geo.stride);
            cudaError_t e = cudaMalloc(&g->links[pi][par], bytes);
            if (e != cudaSuccess) {
                set_error(std::string("wl_gauge_create: cudaMalloc: ") + cudaGetErrorString(e));
                wl_gauge_destroy(g);
                return e == cudaErrorMemoryAllocation ? WL_ERR_OOM : WL_ERR_CUDA;
            }
            dim3 grid((geo.Vh + 127) / 128, 4);
            const double2 *Uc = static_cast<const double2 *>(U);
            if (P == WL_F64) k_pack_links<WL_F64><<<grid, 128, 0, s>>>(geo, Uc, g->links[pi][par], par);
            if (P == WL_F32) k_pack_links<WL_F32><<<grid, 128, 0, s>>>(geo, Uc, g->links[pi][par], par);
            if (P == WL_F16) k_pack_links<WL_F16><<<grid, 128, 0, s>>>(geo, Uc, g->links[pi][par], par);
            if (P == WL_DF) k_pack_links<WL_DF><<<grid, 128, 0, s>>>(geo, Uc, g->links[pi][par], par);
            note_launch(s);
        }
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("wl_gauge_create: ") + cudaGetErrorString(e));
        wl_gauge_destroy(g);
        return WL_ERR_CUDA;
    }
    *out = g;
    return WL_OK;
}

extern "C" int wl_gauge_destroy(wl_gauge *g)
{
    if (!g) return WL_OK;
    cudaDeviceSynchronize();
    for (int pi = 0; pi < 4; ++pi)
        for (int par = 0; par < 2; ++par)
            if (g->links[pi][par]) cudaFree(g->links[pi][par]);
    g->inner_graph.release();
    g->ws.release();
    g->pinned.release();
    delete g;
    return WL_OK;
}
