// Hop kernel instantiations for F64 (one translation unit per precision so the
// library builds in parallel).  Variant v = 100 * (rhs per thread) + (minimum resident
// blocks per SM requested from the register allocator); v = 7000 + 100 * (rhs per
// thread) + B is the grid-stride form with B blocks per SM (k_hop_gs).
#include "hop.cuh"

namespace wl {


template <>
int hop_launch_prec<WL_F64>(int v, int dagger, const HopArgs &a, const EpiStore &e, cudaStream_t s)
{
    if (dagger) {
        switch (v / 100) {
        case 1: launch_k_hop<WL_F64, true, 1, 1>(a, e, s); break;
        case 2: launch_k_hop<WL_F64, true, 2, 1>(a, e, s); break;
        default: launch_k_hop<WL_F64, true, 1, 1>(a, e, s); break;
        }
    } else {
        switch (v) {
        case 101: launch_k_hop<WL_F64, false, 1, 1>(a, e, s); break;
        case 103: launch_k_hop<WL_F64, false, 1, 3>(a, e, s); break;
        case 201: launch_k_hop<WL_F64, false, 2, 1>(a, e, s); break;
        case 7101: launch_k_hop_gs<WL_F64, false, 1, 1>(a, e, s); break;
        case 7102: launch_k_hop_gs<WL_F64, false, 1, 2>(a, e, s); break;
        case 7201: launch_k_hop_gs<WL_F64, false, 2, 1>(a, e, s); break;
        case 7202: launch_k_hop_gs<WL_F64, false, 2, 2>(a, e, s); break;
        default:
            switch (v / 100) {
            case 1: launch_k_hop<WL_F64, false, 1, 1>(a, e, s); break;
            case 2: launch_k_hop<WL_F64, false, 2, 1>(a, e, s); break;
            default: launch_k_hop<WL_F64, false, 1, 1>(a, e, s); break;
            }
        }
    }
    WL_CUDA_TRY(cudaGetLastError());
    return WL_OK;
}

template <>
int hop_reduce_launch_prec<WL_F64>(int kind, int dagger, const HopArgs &a, const void *epi, cudaStream_t s)
{
    switch (kind) {
    case 0: launch_reduce_kind<WL_F64, 0>(dagger, a, epi, s); break;
    case 1: launch_reduce_kind<WL_F64, 1>(dagger, a, epi, s); break;
    case 2: launch_reduce_kind<WL_F64, 2>(dagger, a, epi, s); break;
    default: launch_reduce_kind<WL_F64, 3>(dagger, a, epi, s); break;
    }
    WL_CUDA_TRY(cudaGetLastError());
    return WL_OK;
}

}  // namespace wl
