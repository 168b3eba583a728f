// Host-side internal interfaces between the translation units of libwilson.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <utility>
#include <mutex>
#include <vector>

#include "common.cuh"

struct wl_lattice {
    int dims[4];
    int antiperiodic;
    long volume;
    wl::Geom geom;
};

namespace wl {

// Device buffer owned by the library.
struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
};

// Internal spinor vector (one parity or a batch of rhs of one parity).
struct Vec {
    void *ptr = nullptr;
    int prec = 0;
    int nrhs = 1;
    size_t rhs_bytes = 0;  // bytes between consecutive rhs
    __host__ __device__ void *rhs(int r) const { return static_cast<char *>(ptr) + (size_t)r * rhs_bytes; }
};

// Workspace arena of a gauge handle: named buffers, grown on demand, reused
// across calls, freed with the handle.
struct Workspace {
    std::map<std::string, DevBuf> bufs;
    int get(const std::string &name, size_t bytes, void **out);
    void release();
};

// Page-locked host staging of small per-rhs arrays, by name, kept for the
// life of the handle: cudaMallocHost and cudaFreeHost are slow and may
// synchronise the device, so no solve calls them once the buffers exist.
struct HostPinned {
    std::map<std::string, DevBuf> bufs;
    int get(const std::string &name, size_t bytes, void **out);
    void release();
};




}  // namespace wl

namespace wl {
// Autotuner result for one (precision, rhs count).
struct TuneResult {
    int variant = -1;
    double us = 0.0;
    std::vector<std::pair<int, double>> table;  // every candidate timed (fresh tuning only)
};

// A captured block of inner iterations, reused while its buffers and shape
// are unchanged (the mass enters through device memory).
struct GraphCache {
    std::vector<uintptr_t> key;
    cudaGraphExec_t exec = nullptr;
    long long kernels = 0;
    std::vector<cudaEvent_t> events;
    void release();
};
}  // namespace wl

struct wl_gauge {
    wl::GraphCache inner_graph;
    std::map<std::pair<int, int>, wl::TuneResult> tune;  // (prec, nrhs) -> chosen hop variant
    wl_lattice *lat;
    unsigned prec_mask;
    void *links[4][2];  // [prec index][parity] -> 4 directions of 12-real links
    wl::Workspace ws;
    wl::HostPinned pinned;
    std::mutex mu;      // one solve at a time per handle (shared workspace)
    int profiling = 0;
    wl_kernel_profile prof[4] = {};   // inner hop per precision index (F64, F32, F16); [3] outer residual hop
};

namespace wl {

inline int prec_index(int prec)
{
    return prec == WL_F64 ? 0 : prec == WL_F32 ? 1 : prec == WL_F16 ? 2 : prec == WL_DF ? 3 : -1;
}
inline bool valid_prec(int prec) { return prec_index(prec) >= 0; }

size_t spinor_bytes(const Geom &g, int prec);
int make_vec(wl_gauge *g, const std::string &name, int prec, int nrhs, Vec *v);

// ---- layout.cu
int import_spinors(const Geom &g, const void *const *canon, const Vec &out, int parity, cudaStream_t s);
int export_spinors(const Geom &g, const Vec &in, void *const *canon, int parity, cudaStream_t s);
// Both parities in one pass, with whole-line canonical accesses.
int import_full(const Geom &g, const void *const *canon, const Vec &even, const Vec &odd, cudaStream_t s);
// max_blocks > 0: at most that many blocks, each looping over tiles.
int export_full(const Geom &g, const Vec &even, const Vec &odd, void *const *canon, cudaStream_t s,
                int max_blocks = 0);

// ---- dslash.cu
// out[r] = a1 * x1[r] + a2 * x2[r] + coef * D_{p,1-p} in[r] for r < nrhs (x1, x2
// optional).  rhs_block = rhs per thread (1, 2 or 4).  skip (optional, device)
// skips rhs r when skip[r * skip_stride] != 0.
int hop_ex(wl_gauge *g, const Vec &in, const Vec &out, const Vec *x1, double a1, const Vec *x2, double a2,
           double coef, int out_parity, int dagger, int rhs_block, const int *skip, int skip_stride, cudaStream_t s,
           const Vec *out_raw = nullptr);
int hop(wl_gauge *g, const Vec &in, const Vec &out, const Vec *x, double coef, int out_parity, int dagger,
        int rhs_block, cudaStream_t s);

// Fused solver hops: second half of an operator application followed by the
// BiCGstab reductions; blk_off / blk_total place this launch's blocks in a
// reduction spread over several launches (full-lattice vectors).
//   kind 0:  v = a1 * xin + coef * D tmp;  <rhat, v>        -> alpha = rho / <rhat, v>
//   kind 1:  t = a1 * xin + coef * D tmp;  <t, xin>, <t, t> -> omega
// coef_dev (optional, device) overrides coef at run time.
int hop_reduce(wl_gauge *g, int kind, const Vec &tmp, const Vec &xin, double a1, const Vec &out, const Vec &rhat,
               double coef, const double *coef_dev, int out_parity, int dagger, BiState *state, double *partials,
               int blk_off, int blk_total, cudaStream_t s);

// ---- blas.cu (all on one parity; nrhs from the vectors)
int blas_s_update(const Geom &g, const Vec &r, const Vec &v, const Vec &s_out, BiState *st, cudaStream_t s);
// CG on the normal equations: x += alpha p, r -= alpha w, ||r||^2 -> stop
int blas_cg_xr(const Geom &g, const Vec &x, const Vec &p, const Vec &w, const Vec &r, BiState *state,
               double *partials, cudaStream_t s);
int blas_xr_update(const Geom &g, const Vec &x, const Vec &p, const Vec &sv, const Vec &t, const Vec &r,
                   const Vec &rhat, BiState *st, double *partials, cudaStream_t s);
int blas_p_update(const Geom &g, const Vec &r, const Vec &p, const Vec &v, BiState *st, cudaStream_t s);
int blas_restart(const Geom &g, const Vec &r64, const Vec &r, const Vec &rhat, const Vec &p, const Vec &x,
                 BiState *state, double *partials, const int *active, const double *delta2, cudaStream_t s);
int blas_accum(const Geom &g, const Vec &e, const Vec &x64, const int *active, cudaStream_t s);
int blas_norm2(const Geom &g, const Vec &a, double *out_dev, double *partials, unsigned *tickets, cudaStream_t s);
// out = sum_j c_j in_j, 1 <= k <= 32 inputs, real coefficients per rhs
// c[r * k + j] (cim_dev is ignored)
int blas_lincomb(const Geom &g, const double *cre_dev, const double *cim_dev, const Vec *const *in, int k,
                 const Vec &out, cudaStream_t s);
// out = sum_{j<k} c1_j in_j and out2 = sum_{j<k2} c2_j in_j in one pass;
// complex_coef: the coefficients are (re, im) pairs, c[2 * (r * k + j) + {0, 1}]
// x = sum_j c_j x_j and r = b_prec - x + sum_j d_j y_j in one pass;
// in = x_0..x_{k-1}, y_0..y_{k-1}, b_prec (k <= 15).
int blas_guess_residual(const Geom &g, const double *c_dev, const double *d_dev, const Vec *const *in, int k,
                        const Vec &x, const Vec &r, cudaStream_t s, bool complex_coef);
int blas_lincomb2(const Geom &g, const double *c1_dev, const Vec *const *in, int k, const Vec *out,
                  const double *c2_dev, int k2, const Vec *out2, cudaStream_t s, bool complex_coef = false);
// For each rhs r: dots[r][j] = <in_j[r], a[r]> (j < n, n <= 16), FP64 sums
// over n_complex entries of canonical complex128 arrays; dots_dev holds
// 2 * n * nrhs doubles (re, im).  partials: 2 * 16 * 1024 doubles, tickets: nrhs.
int canon_dots(const void *const *a, const void *const *in, int n, int nrhs, size_t n_complex, double *dots_dev,
               double *partials, unsigned *tickets, cudaStream_t s);
int blas_convert(const Geom &g, const Vec &in, const Vec &out, cudaStream_t s);
int blas_xpay(const Geom &g, const Vec &x, double a, const Vec &y, const Vec &out, cudaStream_t s);  // out = x + a y
// x_o = b_o + kappa Dx and ||b_o - x_o + kappa Dx||^2 per rhs into norm2_dev
int blas_recon(const Geom &g, const Vec &bo, const Vec &dx, double kappa, const Vec &xo, double *norm2_dev,
               double *partials, unsigned *tickets, cudaStream_t s);


// ---- persistent.cu
int persistent_inner(wl_gauge *g, int prec, int nrhs, const Vec &r, const Vec &rhat, const Vec &p, const Vec &v,
                     const Vec &sv, const Vec &t, const Vec &tmp, const Vec &e, BiState *state, const double *kappa2,
                     int max_iter, double deadline_s, int skip_arrival, cudaStream_t s);

// ---- tune.cu
// Hop variant for (prec, nrhs): rhs_block > 0 forces rhs_block rhs per
// thread; rhs_block < 0 selects variant -rhs_block; 0 takes the tuned one.
const std::vector<int> &hop_variants(int prec);
int hop_variant_for(wl_gauge *g, int prec, int nrhs, int rhs_block);
// Bounded device waits (TMA-staged hops) that gave up since the last reset.
int wait_faults(unsigned *count, bool reset, cudaStream_t s);

// Bounds-checked build: status of a synchronising C-ABI call, replaced by
// WL_ERR_CHECKED when an out-of-range site index was recorded (the words are
// left set for wl_checked_status).  The ordinary build returns status as is.
inline int checked_result(int status)
{
#ifdef WL_CHECKED
    unsigned long long v = 0;
    if (checked_status(&v, false) == WL_OK && v) {
        set_error("bounds-checked build: out-of-range site index " + std::to_string(v & 0xffffffffull) +
                  " (access kind " + std::to_string((v >> 32) & 0xff) + ")");
        return WL_ERR_CHECKED;
    }
#endif
    return status;
}
int autotune_hop(wl_gauge *g, int prec, int nrhs, cudaStream_t s, TuneResult *out);

// ---- solver.cu
int full_relres(wl_gauge *g, const Vec &be, const Vec &bo, const Vec &xe, const Vec &xo, double kappa,
                const std::vector<double> &bnorm, std::vector<double> &relres, cudaStream_t s,
                const std::vector<double> *ro_norm2 = nullptr);

}  // namespace wl
