// wilson_dslash_noalloc: the operator application of wilson_dslash for
// callers that must not allocate device memory.
//
// wilson_dslash converts its canonical input and output through four
// internal half-lattice spinors, which it takes from the gauge handle's
// workspace; the first call for a lattice and precision allocates that
// workspace with cudaMalloc.  Some callers cannot let that happen: code that
// runs while another component owns the allocator (a framework's caching
// allocator with a hard memory cap, a memory pool that must not fragment, a
// real-time loop that must not block on cudaMalloc's implicit
// synchronisation).  This variant uses a fixed scratch array that lives in
// the library image instead, so it calls no cudaMalloc, cudaFree or
// allocating library routine.
//
// The scratch is a file-scope __device__ array of kScratchBytes (64 MiB),
// held by every GPU that loads the library until the process exits.  Calls
// share it and it keeps the last call's contents, so two calls whose work
// overlaps on the GPU (different streams, or different host threads) race
// on it; order them on one stream.
#include <mutex>

#include "internal.h"

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  The host-side
// symbol is only a stand-in, so the address is looked up once per device,
// with that device current, and cached.  cudaDeviceReset (or anything else
// that destroys the primary context) unloads the module, so the cached
// address is stale afterwards; the library does not support calls after a
// device reset.
int scratch_address(void **out)
{
    int dev = 0;
    WL_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        wl::set_error("wilson_dslash_noalloc: device index out of range");
        return WL_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        WL_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return WL_OK;
}

}  // namespace

using namespace wl;

extern "C" int wilson_dslash_noalloc(wl_gauge *g, const void *in, void *out, double kappa, int prec, int op,
                                     int dagger, void *stream)
{
    if (!g || !in || !out || in == out || !valid_prec(prec) || op < WL_OP_HOP || op > WL_OP_MPREC) {
        set_error("wilson_dslash_noalloc: bad argument");
        return WL_ERR_ARG;
    }
    if (!(g->prec_mask & prec) || !g->links[prec_index(prec)][0]) {
        set_error("wilson_dslash_noalloc: gauge handle holds no links of the requested precision");
        return WL_ERR_ARG;
    }
    const Geom &geo = g->lat->geom;
    const size_t vec = (spinor_bytes(geo, prec) + 255) & ~(size_t)255;
    if (4 * vec > kScratchBytes) {
        set_error("wilson_dslash_noalloc: lattice too large for the 64 MiB scratch array (needs " +
                  std::to_string(4 * vec) + " bytes: four half-lattice spinors of this precision)");
        return WL_ERR_ARG;
    }
    void *base = nullptr;
    WL_TRY(scratch_address(&base));
    // the hop variant lookup reads the handle's tuning table, which
    // wl_autotune may be filling from another thread
    std::lock_guard<std::mutex> lock(g->mu);
    cudaStream_t s = as_stream(stream);
    Vec ie, io, oe, oo;
    Vec *v[4] = {&ie, &io, &oe, &oo};
    for (int k = 0; k < 4; ++k) {
        v[k]->ptr = static_cast<char *>(base) + k * vec;
        v[k]->prec = prec;
        v[k]->nrhs = 1;
        v[k]->rhs_bytes = vec;
    }
    const int dag = dagger ? 1 : 0;
    const void *cin[1] = {in};
    void *cout[1] = {out};
    // every scratch buffer is fully written below before it is read, except
    // the odd output of M_prec, which is defined as zero
    WL_TRY(import_full(geo, cin, ie, io, s));
    if (op == WL_OP_HOP) {
        WL_TRY(hop(g, io, oe, nullptr, 1.0, WL_EVEN, dag, 1, s));
        WL_TRY(hop(g, ie, oo, nullptr, 1.0, WL_ODD, dag, 1, s));
    } else if (op == WL_OP_M) {
        WL_TRY(hop(g, io, oe, &ie, -kappa, WL_EVEN, dag, 1, s));
        WL_TRY(hop(g, ie, oo, &io, -kappa, WL_ODD, dag, 1, s));
    } else {
        WL_TRY(hop(g, ie, oo, nullptr, 1.0, WL_ODD, dag, 1, s));
        WL_TRY(hop(g, oo, oe, &ie, -kappa * kappa, WL_EVEN, dag, 1, s));
        WL_CUDA_TRY(cudaMemsetAsync(oo.ptr, 0, spinor_bytes(geo, prec), s));
    }
    WL_TRY(export_full(geo, oe, oo, cout, s));
    return WL_OK;
}
