// Internal types and device helpers shared by the CUDA translation units of
// libwilson.  Not part of the C ABI.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "wilson.h"

namespace wl {

// ------------------------------------------------------------------ errors

void set_error(const std::string &msg);

#define WL_CUDA_TRY(expr)                                                                   \
    do {                                                                                    \
        cudaError_t _e = (expr);                                                            \
        if (_e != cudaSuccess) {                                                            \
            ::wl::set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));            \
            return _e == cudaErrorMemoryAllocation ? WL_ERR_OOM : WL_ERR_CUDA;              \
        }                                                                                   \
    } while (0)

#define WL_TRY(expr)                  \
    do {                              \
        int _s = (expr);              \
        if (_s != WL_OK) return _s;   \
    } while (0)

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// ----------------------------------------------------- bounds-checked build
// With WL_CHECKED defined (libwilson_checked.so, built beside the library)
// every site index of an internal spinor or link access is tested against
// the length of its array.  The first violation in each translation unit
// is recorded in a device word -- bit 63 set, the access kind (1 spinor
// load, 2 spinor store, 3 link load) in bits 32-39, the index in bits 0-31
// -- and the access goes to site 0 (a load) or is dropped (a store), so
// nothing outside the arrays is touched and nothing traps.  The C-ABI calls
// that synchronise return WL_ERR_CHECKED when a word is set;
// wl_checked_status reads and clears them.  In the ordinary build the
// checks compile to nothing.
int checked_register(int (*reader)(unsigned long long *, bool));
int checked_status(unsigned long long *first, bool reset);

#ifdef WL_CHECKED
namespace checked {
static __device__ unsigned long long first_violation;   // one per translation unit
}
__device__ __forceinline__ bool in_range(int i, int n, unsigned kind)
{
    if ((unsigned)i < (unsigned)n) return true;
    atomicCAS(&checked::first_violation, 0ull, (1ull << 63) | ((unsigned long long)kind << 32) | (unsigned)i);
    return false;
}
#define WL_LOAD_IDX(i, n, kind) (::wl::in_range((i), (n), (kind)) ? (i) : 0)
#define WL_STORE_OK(i, n, kind) ::wl::in_range((i), (n), (kind))
namespace checked {
static int read_word(unsigned long long *v, bool reset)
{
    WL_CUDA_TRY(cudaMemcpyFromSymbol(v, first_violation, sizeof(unsigned long long)));
    if (reset && *v) {
        const unsigned long long zero = 0;
        WL_CUDA_TRY(cudaMemcpyToSymbol(first_violation, &zero, sizeof(unsigned long long)));
    }
    return WL_OK;
}
static const int registered = checked_register(&read_word);
}  // namespace checked
#else
#define WL_LOAD_IDX(i, n, kind) (i)
#define WL_STORE_OK(i, n, kind) true
#endif

// Kernel launch accounting (wl_launch_count): note_launch(s) after a launch
// on stream s counts it unless s is being captured into a graph; graph
// replays add their kernel-node count through add_launches.
void note_launch(cudaStream_t s);
void add_launches(long long n);

// ---------------------------------------------------------------- geometry

// Lattice geometry in the form the kernels need.  Sites of one parity are
// numbered i = floor(lex / 2) with lex = x + X*(y + Y*(z + Z*t)) (Section 4:
// even sites first, then odd; within a parity, lexicographic order).
struct Geom {
    int X, Y, Z, T;
    int Xh;          // X / 2
    int Vh;          // sites per parity
    int stride;      // padded per-parity array length (multiple of 64)
    int antiperiodic;
};

// Coordinates of site i of parity p.
struct Coord {
    int x, y, z, t;
};

__device__ __forceinline__ Coord site_coord(const Geom &g, int i, int p)
{
    Coord c;
    int xh = i % g.Xh;
    int r = i / g.Xh;
    c.y = r % g.Y;
    r /= g.Y;
    c.z = r % g.Z;
    c.t = r / g.Z;
    c.x = 2 * xh + ((p + c.y + c.z + c.t) & 1);
    return c;
}

// Per-parity index of the site with coordinates c (either parity).
__device__ __forceinline__ int site_index(const Geom &g, int x, int y, int z, int t)
{
    return (x >> 1) + g.Xh * (y + g.Y * (z + g.Z * t));
}

// ------------------------------------------------------------------ complex

template <typename R>
struct cx {
    R re, im;
};

template <typename R>
__device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R>
__device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R>
__device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b)
{
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R>
__device__ __forceinline__ cx<R> operator*(R s, cx<R> a) { return {s * a.re, s * a.im}; }
template <typename R>
__device__ __forceinline__ cx<R> conjmul(cx<R> a, cx<R> b)  // conj(a) * b
{
    return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
template <typename R>
__device__ __forceinline__ cx<R> cmad(cx<R> a, cx<R> b, cx<R> c)  // a*b + c
{
    return {fma(a.re, b.re, fma(-a.im, b.im, c.re)), fma(a.re, b.im, fma(a.im, b.re, c.im))};
}
template <typename R>
__device__ __forceinline__ cx<R> conjmad(cx<R> a, cx<R> b, cx<R> c)  // conj(a)*b + c
{
    return {fma(a.re, b.re, fma(a.im, b.im, c.re)), fma(a.re, b.im, fma(-a.im, b.re, c.im))};
}

// ------------------------------------------------------------ double-float
//
// A double-float value is the unevaluated sum hi + lo of two FP32 numbers
// with |lo| <= ulp(hi)/2, about 48 significant bits.  GB300 executes FP64 at
// 1/57 of its FP32 rate, so the FP64-class parts of the solver (residual
// recomputation, solution accumulator, even-odd reconstruction) run in this
// format on the FP32 pipes.  The operations are the classical error-free
// transformations: Knuth's two-sum, the FMA two-product, and Dekker's
// renormalisation (fast two-sum); products and sums keep the low-order
// cross terms, so the relative error of each operation is a few 2^-48.

struct df {
    float hi, lo;
    __host__ __device__ df() {}
    __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ explicit constexpr df(int v) : hi((float)v), lo(0.f) {}
    __host__ __device__ explicit constexpr df(float v) : hi(v), lo(0.f) {}
    // split a double: hi = round(d), lo = round(d - hi)
    __host__ __device__ explicit df(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
};

using ::fma;  // keep the float/double overloads visible next to the df one

// The error-free transformations below must be evaluated exactly as
// written: the compiler may otherwise contract a product with a later sum
// into one FMA, which changes the rounding the error terms assume.  The
// __fmul_rn / __fadd_rn / __fsub_rn intrinsics are never contracted.
__device__ __forceinline__ df df_fast_two_sum(float a, float b)  // |a| >= |b|
{
    const float s = __fadd_rn(a, b);
    return df(s, __fsub_rn(b, __fsub_rn(s, a)));
}

// Arithmetic results are kept "lazy": the low word collects the exact
// rounding error of the high operation plus the low-order terms, without the
// final renormalisation; |lo| stays within a few ulp(hi), so further
// operations lose nothing measurable, and SpinorIO<WL_DF>::store
// renormalises before anything is written to memory.
__device__ __forceinline__ df operator+(df a, df b)
{
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    // Knuth two-sum error of the high parts
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    return df(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator*(df a, df b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);  // exact error of the high product
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df(p, e);
}
__device__ __forceinline__ df df_normalize(df a) { return df_fast_two_sum(a.hi, a.lo); }
__device__ __forceinline__ df fma(df a, df b, df c) { return a * b + c; }
__device__ __forceinline__ double to_double(df a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ double to_double(float a) { return (double)a; }
__device__ __forceinline__ double to_double(double a) { return a; }
__device__ __forceinline__ float to_float(df a) { return a.hi + a.lo; }

// Conversions between arithmetic types (double <-> df go through the split).
template <typename T> struct Conv;
template <> struct Conv<double> {
    static __device__ __forceinline__ double from(double v) { return v; }
    static __device__ __forceinline__ double from(float v) { return (double)v; }
    static __device__ __forceinline__ double from(df v) { return to_double(v); }
};
template <> struct Conv<float> {
    static __device__ __forceinline__ float from(double v) { return (float)v; }
    static __device__ __forceinline__ float from(float v) { return v; }
    static __device__ __forceinline__ float from(df v) { return to_float(v); }
};
template <> struct Conv<df> {
    static __device__ __forceinline__ df from(double v) { return df(v); }
    static __device__ __forceinline__ df from(float v) { return df(v); }
    static __device__ __forceinline__ df from(df v) { return v; }
};

// ---------------------------------------------------------- precision I/O

// Arithmetic type per storage precision: FP16 storage computes in FP32.
template <int P> struct PrecTraits;
template <> struct PrecTraits<WL_F64> { using R = double; };
template <> struct PrecTraits<WL_F32> { using R = float; };
template <> struct PrecTraits<WL_F16> { using R = float; };
template <> struct PrecTraits<WL_DF> { using R = df; };

// Bytes per site of an internal spinor / per site of one direction's link.
__host__ __device__ constexpr int spinor_site_bytes(int prec)
{
    return prec == WL_F64 ? 192 : prec == WL_F32 ? 96 : prec == WL_DF ? 192 : 52;
}
__host__ __device__ constexpr int link_site_bytes(int prec)
{
    return prec == WL_F64 ? 144 : prec == WL_F32 ? 48 : prec == WL_DF ? 144 : 36;
}

// Start value of every hop accumulator: -0.0.  x + (-0.0) == x exactly for
// every x (+0 and -0 included), so the compiler may turn the first
// accumulation into each output component into a move; with +0.0 it may
// not (+0 + -0 is +0), and the first of the eight transporters would cost
// 24 adds per site and rhs.
template <typename R>
__device__ __forceinline__ cx<R> acc_zero()
{
    return {R(-0.0f), R(-0.0f)};
}

// Squared magnitude accumulated per site: FP32 for FP32 and double-float
// data (high words only -- a relative 2^-23 on a norm is plenty for
// stopping tests and reported residuals), FP64 for FP64 data.  Sites are
// then summed in FP64.
__device__ __forceinline__ void norm_acc(float &n, float x) { n = fmaf(x, x, n); }
__device__ __forceinline__ void norm_acc(float &n, df x)
{
    const float v = x.hi + x.lo;  // lazy values may have |lo| ~ |hi|: square the sum, never negative
    n = fmaf(v, v, n);
}
__device__ __forceinline__ void norm_acc(double &n, double x) { n = fma(x, x, n); }
template <typename R> struct NormT { using T = float; };
template <> struct NormT<double> { using T = double; };

// Vector loads: the read-only path (__ldg) for data that no block of the
// running kernel writes; ordinary loads for data that other blocks of the
// same (persistent) kernel rewrite between grid barriers -- after the
// barrier's release/acquire fences those are coherent, the non-coherent
// read-only path is not.
template <bool CG, typename T>
__device__ __forceinline__ T ldx(const T *p)
{
    if constexpr (CG) return *p;
    else return __ldg(p);
}

template <typename To, typename From>
__device__ __forceinline__ cx<To> cconv(cx<From> z)
{
    return {Conv<To>::from(z.re), Conv<To>::from(z.im)};
}

// Internal spinor layout, component k = 3*spin + colour (12 complex):
//   F64: double2 [12][stride]
//   F32: float4  [6][stride]   (chunk j = components 2j, 2j+1)
//   F16: uint4   [3][stride]   (chunk j = components 4j..4j+3 as half2)
//        followed by float norm[stride]; value = half * norm.
//   DF:  float4  [12][stride]  (chunk k = component k as re.hi, re.lo, im.hi, im.lo)
template <int P> struct SpinorIO;

// load_unscaled(base, stride, i, v) returns a factor f with site value =
// f * v: the per-site norm for FP16 storage (v the unscaled halves), 1 for
// the other formats (v the values).
template <> struct SpinorIO<WL_F64> {
    using R = double;
    template <bool CG = false>
    static __device__ __forceinline__ void load(const void *base, int stride, int i, cx<R> (&v)[12])
    {
        i = WL_LOAD_IDX(i, stride, 1);
        const double2 *p = static_cast<const double2 *>(base);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            double2 t = ldx<CG>(p + (size_t)k * stride + i);
            v[k] = {t.x, t.y};
        }
    }
    template <bool CG = false>
    static __device__ __forceinline__ R load_unscaled(const void *base, int stride, int i, cx<R> (&v)[12])
    {
        load<CG>(base, stride, i, v);
        return 1.0;
    }
    static __device__ __forceinline__ void roundtrip(cx<R> (&)[12]) {}
    static __device__ __forceinline__ void store_rounded(void *base, int stride, int i, cx<R> (&v)[12])
    {
        store(base, stride, i, v);
    }
    static __device__ __forceinline__ void store(void *base, int stride, int i, const cx<R> (&v)[12])
    {
        if (!WL_STORE_OK(i, stride, 2)) return;
        double2 *p = static_cast<double2 *>(base);
#pragma unroll
        for (int k = 0; k < 12; ++k) p[(size_t)k * stride + i] = make_double2(v[k].re, v[k].im);
    }
};

template <> struct SpinorIO<WL_F32> {
    using R = float;
    template <bool CG = false>
    static __device__ __forceinline__ void load(const void *base, int stride, int i, cx<R> (&v)[12])
    {
        i = WL_LOAD_IDX(i, stride, 1);
        const float4 *p = static_cast<const float4 *>(base);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            float4 t = ldx<CG>(p + (size_t)k * stride + i);
            v[2 * k] = {t.x, t.y};
            v[2 * k + 1] = {t.z, t.w};
        }
    }
    template <bool CG = false>
    static __device__ __forceinline__ R load_unscaled(const void *base, int stride, int i, cx<R> (&v)[12])
    {
        load<CG>(base, stride, i, v);
        return 1.f;
    }
    static __device__ __forceinline__ void roundtrip(cx<R> (&)[12]) {}
    static __device__ __forceinline__ void store_rounded(void *base, int stride, int i, cx<R> (&v)[12])
    {
        store(base, stride, i, v);
    }
    static __device__ __forceinline__ void store(void *base, int stride, int i, const cx<R> (&v)[12])
    {
        if (!WL_STORE_OK(i, stride, 2)) return;
        float4 *p = static_cast<float4 *>(base);
#pragma unroll
        for (int k = 0; k < 6; ++k)
            p[(size_t)k * stride + i] = make_float4(v[2 * k].re, v[2 * k].im, v[2 * k + 1].re, v[2 * k + 1].im);
    }
};

__device__ __forceinline__ uint32_t pack_half2(float a, float b)
{
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}
__device__ __forceinline__ float2 unpack_half2(uint32_t u)
{
    __half2 h = *reinterpret_cast<__half2 *>(&u);
    return __half22float2(h);
}

template <> struct SpinorIO<WL_F16> {
    using R = float;
    // Per-site scale = max |component|.  A site whose largest entry is below
    // the smallest normal float is stored as zero: 1/scale would overflow to
    // inf there (and 0 * inf = NaN), and such a site is below 1e-38 of any
    // unit-normalised vector.  Point-source residuals decay exponentially
    // with distance and reach this range on large lattices.
    static __device__ __forceinline__ float site_scale(const cx<R> (&v)[12])
    {
        float m = 0.f;
#pragma unroll
        for (int k = 0; k < 12; ++k) m = fmaxf(m, fmaxf(fabsf(v[k].re), fabsf(v[k].im)));
        return m >= 1.17549435e-38f ? m : 0.f;
    }
    static __device__ __forceinline__ const float *norms(const void *base, int stride)
    {
        return reinterpret_cast<const float *>(static_cast<const uint4 *>(base) + 3 * (size_t)stride);
    }
    template <bool CG = false>
    static __device__ __forceinline__ R load_unscaled(const void *base, int stride, int i, cx<R> (&v)[12])
    {
        i = WL_LOAD_IDX(i, stride, 1);
        const uint4 *p = static_cast<const uint4 *>(base);
        const float n = ldx<CG>(norms(base, stride) + i);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint4 t = ldx<CG>(p + (size_t)k * stride + i);
            float2 a = unpack_half2(t.x), b = unpack_half2(t.y), c = unpack_half2(t.z), d = unpack_half2(t.w);
            v[4 * k + 0] = {a.x, a.y};
            v[4 * k + 1] = {b.x, b.y};
            v[4 * k + 2] = {c.x, c.y};
            v[4 * k + 3] = {d.x, d.y};
        }
        return n;
    }
    template <bool CG = false>
    static __device__ __forceinline__ void load(const void *base, int stride, int i, cx<R> (&v)[12])
    {
        i = WL_LOAD_IDX(i, stride, 1);
        const uint4 *p = static_cast<const uint4 *>(base);
        const float n = ldx<CG>(norms(base, stride) + i);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint4 t = ldx<CG>(p + (size_t)k * stride + i);
            float2 a = unpack_half2(t.x), b = unpack_half2(t.y), c = unpack_half2(t.z), d = unpack_half2(t.w);
            v[4 * k + 0] = {a.x * n, a.y * n};
            v[4 * k + 1] = {b.x * n, b.y * n};
            v[4 * k + 2] = {c.x * n, c.y * n};
            v[4 * k + 3] = {d.x * n, d.y * n};
        }
    }
    static __device__ __forceinline__ void store(void *base, int stride, int i, const cx<R> (&v)[12])
    {
        if (!WL_STORE_OK(i, stride, 2)) return;
        float m = site_scale(v);
        const float inv = m > 0.f ? 1.0f / m : 0.f;
        uint4 *p = static_cast<uint4 *>(base);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint4 t;
            t.x = pack_half2(v[4 * k + 0].re * inv, v[4 * k + 0].im * inv);
            t.y = pack_half2(v[4 * k + 1].re * inv, v[4 * k + 1].im * inv);
            t.z = pack_half2(v[4 * k + 2].re * inv, v[4 * k + 2].im * inv);
            t.w = pack_half2(v[4 * k + 3].re * inv, v[4 * k + 3].im * inv);
            p[(size_t)k * stride + i] = t;
        }
        const_cast<float *>(norms(base, stride))[i] = m;
    }
    // Replace v by the values a store followed by a load would return.
    static __device__ __forceinline__ void roundtrip(cx<R> (&v)[12])
    {
        const float m = site_scale(v);
        const float inv = m > 0.f ? 1.0f / m : 0.f;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            float2 h = unpack_half2(pack_half2(v[k].re * inv, v[k].im * inv));
            v[k] = {h.x * m, h.y * m};
        }
    }
    // store, and replace v by the stored values (one scale and one packing
    // for both)
    static __device__ __forceinline__ void store_rounded(void *base, int stride, int i, cx<R> (&v)[12])
    {
        if (!WL_STORE_OK(i, stride, 2)) return;
        const float m = site_scale(v);
        const float inv = m > 0.f ? 1.0f / m : 0.f;
        uint32_t w[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            w[k] = pack_half2(v[k].re * inv, v[k].im * inv);
            const float2 h = unpack_half2(w[k]);
            v[k] = {h.x * m, h.y * m};
        }
        uint4 *p = static_cast<uint4 *>(base);
#pragma unroll
        for (int k = 0; k < 3; ++k) p[(size_t)k * stride + i] = make_uint4(w[4 * k], w[4 * k + 1], w[4 * k + 2], w[4 * k + 3]);
        const_cast<float *>(norms(base, stride))[i] = m;
    }
};

template <> struct SpinorIO<WL_DF> {
    using R = df;
    template <bool CG = false>
    static __device__ __forceinline__ void load(const void *base, int stride, int i, cx<R> (&v)[12])
    {
        i = WL_LOAD_IDX(i, stride, 1);
        const float4 *p = static_cast<const float4 *>(base);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            float4 t = ldx<CG>(p + (size_t)k * stride + i);
            v[k] = {df(t.x, t.y), df(t.z, t.w)};
        }
    }
    template <bool CG = false>
    static __device__ __forceinline__ R load_unscaled(const void *base, int stride, int i, cx<R> (&v)[12])
    {
        load<CG>(base, stride, i, v);
        return df(1.f);
    }
    static __device__ __forceinline__ void roundtrip(cx<R> (&)[12]) {}
    static __device__ __forceinline__ void store_rounded(void *base, int stride, int i, cx<R> (&v)[12])
    {
        store(base, stride, i, v);
    }
    static __device__ __forceinline__ void store(void *base, int stride, int i, const cx<R> (&v)[12])
    {
        if (!WL_STORE_OK(i, stride, 2)) return;
        float4 *p = static_cast<float4 *>(base);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const df re = df_normalize(v[k].re), im = df_normalize(v[k].im);
            p[(size_t)k * stride + i] = make_float4(re.hi, re.lo, im.hi, im.lo);
        }
    }
};

// Links: per parity, per direction (k = 3*row + col):
//   F32: float4 [4][3][stride]  (rows 0-1, 6 complex; row 2 is rebuilt as
//        conj(row0 x row1))
//   F16: per direction uint2 [4][stride] (entries 0-7 as half2 pairs) then
//        uint [stride] (entry 8): all three rows, 36 bytes per site
//   F64: double2 [4][9][stride]  (all three rows)
//   DF:  float4 [4][9][stride] (re.hi, re.lo, im.hi, im.lo), all three rows
template <int P> struct LinkIO;

template <typename R>
__device__ __forceinline__ void reconstruct_row2(cx<R> (&u)[9])
{
    // u[6+c] = conj(r0 x r1)_c
    cx<R> a = u[1] * u[5] - u[2] * u[4];
    cx<R> b = u[2] * u[3] - u[0] * u[5];
    cx<R> c = u[0] * u[4] - u[1] * u[3];
    u[6] = {a.re, -a.im};
    u[7] = {b.re, -b.im};
    u[8] = {c.re, -c.im};
}

// FP64 links keep all three rows as given (18 reals): the FP64 hop is bound
// by the FP64 pipe (1/57 of the FP32 rate on GB300), where rebuilding row 2
// costs about 10% of its instructions, and not by memory, where the extra
// 48 B per link are cheap.
template <> struct LinkIO<WL_F64> {
    using R = double;
    static constexpr int chunks = 9;
    static __device__ __forceinline__ void load(const void *dirbase, int stride, int i, cx<R> (&u)[9])
    {
        i = WL_LOAD_IDX(i, stride, 3);
        const double2 *p = static_cast<const double2 *>(dirbase);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            double2 t = __ldg(p + (size_t)k * stride + i);
            u[k] = {t.x, t.y};
        }
    }
};
template <> struct LinkIO<WL_F32> {
    using R = float;
    static constexpr int chunks = 3;
    // rows 0 and 1 only (u[0..5])
    static __device__ __forceinline__ void load_rows(const void *dirbase, int stride, int i, cx<R> (&u)[9])
    {
        i = WL_LOAD_IDX(i, stride, 3);
        const float4 *p = static_cast<const float4 *>(dirbase);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float4 t = __ldg(p + (size_t)k * stride + i);
            u[2 * k] = {t.x, t.y};
            u[2 * k + 1] = {t.z, t.w};
        }
    }
    static __device__ __forceinline__ void load(const void *dirbase, int stride, int i, cx<R> (&u)[9])
    {
        load_rows(dirbase, stride, i, u);
        reconstruct_row2(u);
    }
};
// FP16 links keep row 2 as well (12 bytes more per link): the FP16 hop is
// bound by instruction issue and the FMA pipe, where rebuilding row 2 costs
// about a fifth of its FMA work, and not by memory.
template <> struct LinkIO<WL_F16> {
    using R = float;
    static constexpr int chunks = 3;
    // rows 0 and 1 only (u[0..5])
    static __device__ __forceinline__ void load_rows(const void *dirbase, int stride, int i, cx<R> (&u)[9])
    {
        i = WL_LOAD_IDX(i, stride, 3);
        const uint2 *p = static_cast<const uint2 *>(dirbase);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint2 t = __ldg(p + (size_t)k * stride + i);
            float2 a = unpack_half2(t.x), b = unpack_half2(t.y);
            u[2 * k] = {a.x, a.y};
            u[2 * k + 1] = {b.x, b.y};
        }
    }
    static __device__ __forceinline__ void load(const void *dirbase, int stride, int i, cx<R> (&u)[9])
    {
        load_rows(dirbase, stride, i, u);
        i = WL_LOAD_IDX(i, stride, 3);
        const uint2 t = __ldg(static_cast<const uint2 *>(dirbase) + (size_t)3 * stride + i);
        const unsigned w = __ldg(reinterpret_cast<const unsigned *>(static_cast<const uint2 *>(dirbase) + (size_t)4 * stride) + i);
        const float2 a = unpack_half2(t.x), b = unpack_half2(t.y), c = unpack_half2(w);
        u[6] = {a.x, a.y};
        u[7] = {b.x, b.y};
        u[8] = {c.x, c.y};
    }
};

// Double-float links keep all three rows (18 reals): rebuilding row 2 in
// double-float arithmetic costs about 14% of the double-float hop's
// instructions, while the extra 48 B per link are free in a hop that is
// bound by instruction issue, not by memory.  Row 2 is formed once in FP64
// when the links are packed.
template <> struct LinkIO<WL_DF> {
    using R = df;
    static constexpr int chunks = 9;
    static __device__ __forceinline__ void load(const void *dirbase, int stride, int i, cx<R> (&u)[9])
    {
        i = WL_LOAD_IDX(i, stride, 3);
        const float4 *p = static_cast<const float4 *>(dirbase);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            float4 t = __ldg(p + (size_t)k * stride + i);
            u[k] = {df(t.x, t.y), df(t.z, t.w)};
        }
    }
};

// Byte offset of direction mu inside one parity's link block.
__host__ __device__ inline size_t link_dir_bytes(int prec, int stride)
{
    return (size_t)link_site_bytes(prec) * stride;
}

// ---------------------------------------------------------------- reductions

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of NV doubles per thread; result valid in thread 0.
// Fixed tree order (deterministic).  blockDim.x must be a multiple of 32, <= 1024.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV])
{
    __shared__ double sh[32][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[warp][k] = v[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double t = lane < nw ? sh[lane][k] : 0.0;
            v[k] = warp_sum(t);
        }
    }
    __syncthreads();
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of NV FP32 values per thread, result in FP64 (valid in
// thread 0): FP32 inside the block, converted once (blocks then combine in
// FP64).  The per-thread values are FP32 partials over one site, so the
// block's few hundred of them summed in FP32 stay in the same accuracy
// class, and GB300 runs FP64 arithmetic at 1/57 of the FP32 rate: a warp
// sum of doubles costs each thread five FP64 adds per value, and with them
// the FP64 pipe of the reduction-fused hops was 15% busy.
template <int NV>
__device__ __forceinline__ void block_sum(float (&vf)[NV], double (&v)[NV])
{
    __shared__ float sh[32][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) vf[k] = warp_sum(vf[k]);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[warp][k] = vf[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const float t = lane < nw ? sh[lane][k] : 0.f;
            v[k] = (double)warp_sum(t);
        }
    }
    __syncthreads();
}

// Per-thread reduction type: FP32 partials for FP32 arithmetic (FP16
// storage included), FP64 otherwise (FP64 and double-float data).
template <typename R> struct RedType { using T = double; };
template <> struct RedType<float> { using T = float; };
template <typename T, typename R>
__device__ __forceinline__ T red_cast(R x)
{
    if constexpr (sizeof(T) == sizeof(float)) return x;
    else return to_double(x);
}

// Grid-wide deterministic reduction without a second launch ("last block"
// pattern): every block deposits its NV partial sums in partials[blk][NV];
// the block that arrives last (atomic ticket) adds the partials in block
// order and returns true in all of its threads with the totals in tot
// (valid in thread 0).  The ticket is reset to zero for the next use.
// `nblk` blocks take part, numbered blk = 0..nblk-1.  Per-thread values
// may be FP32 (summed as block_sum above) or FP64; blocks combine in FP64.
template <int NV>
__device__ __forceinline__ bool grid_finish(double (&v)[NV], double *partials, unsigned *ticket, int blk,
                                            int nblk, double (&tot)[NV]);

template <int NV>
__device__ __forceinline__ bool grid_sum(float (&vf)[NV], double *partials, unsigned *ticket, int blk,
                                         int nblk, double (&tot)[NV])
{
    double v[NV];
    block_sum<NV>(vf, v);
    return grid_finish<NV>(v, partials, ticket, blk, nblk, tot);
}

template <int NV>
__device__ __forceinline__ bool grid_sum(double (&v)[NV], double *partials, unsigned *ticket, int blk,
                                         int nblk, double (&tot)[NV])
{
    block_sum<NV>(v);
    return grid_finish<NV>(v, partials, ticket, blk, nblk, tot);
}

template <int NV>
__device__ __forceinline__ bool grid_finish(double (&v)[NV], double *partials, unsigned *ticket, int blk,
                                            int nblk, double (&tot)[NV])
{
    __shared__ bool is_last;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) partials[(size_t)blk * NV + k] = v[k];
        __threadfence();
        unsigned t = atomicAdd(ticket, 1u);
        is_last = (t == (unsigned)nblk - 1);
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    double acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < NV; ++k) acc[k] += __ldcg(partials + (size_t)b * NV + k);
    block_sum<NV>(acc);
#pragma unroll
    for (int k = 0; k < NV; ++k) tot[k] = acc[k];
    if (threadIdx.x == 0) *ticket = 0u;
    return true;
}

// --------------------------------------------------------- solver scalars

// Device-resident BiCGstab scalars of one right-hand side (FP64).  Each
// iteration's kernels read and update these, so no host round trip is
// needed inside an iteration.
struct BiState {
    double rho_re, rho_im;      // <rhat, r>
    double alpha_re, alpha_im;
    double omega_re, omega_im;
    double beta_re, beta_im;
    double rr;                  // ||r||^2 of the latest residual
    double target2;             // stop when rr <= target2
    // Breakdown test: |<rhat, r>|^2 or |<rhat, v>|^2 at or below
    // brk2 * ||rhat||^2 * ||.||^2.  brk2 = 0 (the default) tests for exact zero.
    double rhat2;
    double brk2;
    int done;                   // 1: converged or broken down -> kernels skip this rhs
    int breakdown;              // 1: a denominator vanished
    int iters;                  // completed iterations
    int pad;
    unsigned ticket[4];         // last-block tickets, one per reduction site
};

// Reduction scratch: partials[(rhs * nblocks + block) * kRedNV + k].
constexpr int kRedNV = 4;
constexpr int kBlock = 128;  // threads per block of every site kernel
inline int site_blocks(const Geom &g) { return (g.Vh + kBlock - 1) / kBlock; }

}  // namespace wl
