// Hop kernel instantiations for DF (one translation unit per precision so the
// library builds in parallel).  Variant v = 100 * (rhs per thread) + (minimum resident
// blocks per SM requested from the register allocator).
#include "hop.cuh"

namespace wl {

template <>
int hop_launch_prec<WL_DF>(int v, int dagger, const HopArgs &a, const EpiStore &e, cudaStream_t s)
{
    if (dagger) {
        launch_k_hop_rolled<WL_DF, true, 1>(a, e, s);
    } else {
        switch (v) {
        case 101: launch_k_hop_rolled<WL_DF, false, 1>(a, e, s); break;
        case 103: launch_k_hop_rolled<WL_DF, false, 3>(a, e, s); break;
        case 104: launch_k_hop_rolled<WL_DF, false, 4>(a, e, s); break;
        case 105: launch_k_hop_rolled<WL_DF, false, 5>(a, e, s); break;
        case 106: launch_k_hop_rolled<WL_DF, false, 6>(a, e, s); break;
        default: launch_k_hop_rolled<WL_DF, false, 1>(a, e, s); break;
        }
    }
    WL_CUDA_TRY(cudaGetLastError());
    return WL_OK;
}

template <>
int hop_reduce_launch_prec<WL_DF>(int kind, int dagger, const HopArgs &a, const void *epi, cudaStream_t s)
{
    // double-float BiCGstab-M (kinds 0 and 1 only)
    switch (kind) {
    case 0: launch_reduce_kind<WL_DF, 0>(dagger, a, epi, s); break;
    case 1: launch_reduce_kind<WL_DF, 1>(dagger, a, epi, s); break;
    default: set_error("hop_reduce: double-float supports kinds 0 and 1"); return WL_ERR_ARG;
    }
    WL_CUDA_TRY(cudaGetLastError());
    return WL_OK;
}

}  // namespace wl
