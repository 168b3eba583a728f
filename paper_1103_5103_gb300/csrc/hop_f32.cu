// Hop kernel instantiations for F32 (one translation unit per precision so the
// library builds in parallel).  Variant v = 100 * (rhs per thread) + (minimum resident
// blocks per SM requested from the register allocator); 5006 is the paired-site hop
// (two sites per thread in packed FP32 arithmetic, 64-thread blocks, six resident per
// SM: 168 registers; a tighter budget spills); 9000 + 100 b + R is the TMA-staged hop with R rhs per tile and
// register budget b (hop_tma.cu).
#include "hop.cuh"

namespace wl {

template <>
int hop_launch_prec<WL_F32>(int v, int dagger, const HopArgs &a, const EpiStore &e, cudaStream_t s)
{
    if (v >= 9000 && v < 9300 && !dagger) {
        const int st = hop_launch_tma(WL_F32, v, dagger, a, e, s);
        if (st != WL_OK) return st;
        WL_CUDA_TRY(cudaGetLastError());
        return WL_OK;
    }
    if (dagger) {
        switch (v / 100) {
        case 1: launch_k_hop<WL_F32, true, 1, 1>(a, e, s); break;
        case 2: launch_k_hop<WL_F32, true, 2, 1>(a, e, s); break;
        case 4: launch_k_hop<WL_F32, true, 4, 1>(a, e, s); break;
        default: launch_k_hop<WL_F32, true, 1, 1>(a, e, s); break;
        }
    } else {
        switch (v) {
        case 1104: launch_k_hop_async<false, 1, 4>(a, e, s); break;
        case 1106: launch_k_hop_async<false, 1, 6>(a, e, s); break;
        case 1202: launch_k_hop_async<false, 2, 2>(a, e, s); break;
        case 1203: launch_k_hop_async<false, 2, 3>(a, e, s); break;
        case 301: launch_k_hop_prefetch_f32<false, 1>(a, e, s); break;
        case 304: launch_k_hop_prefetch_f32<false, 4>(a, e, s); break;
        case 305: launch_k_hop_prefetch_f32<false, 5>(a, e, s); break;
        case 5006: launch_k_hop_pair<WL_F32, false, 6>(a, e, s); break;
        case 101: launch_k_hop<WL_F32, false, 1, 1>(a, e, s); break;
        case 105: launch_k_hop<WL_F32, false, 1, 5>(a, e, s); break;
        case 106: launch_k_hop<WL_F32, false, 1, 6>(a, e, s); break;
        case 108: launch_k_hop<WL_F32, false, 1, 8>(a, e, s); break;
        case 201: launch_k_hop<WL_F32, false, 2, 1>(a, e, s); break;
        case 204: launch_k_hop<WL_F32, false, 2, 4>(a, e, s); break;
        case 205: launch_k_hop<WL_F32, false, 2, 5>(a, e, s); break;
        case 401: launch_k_hop<WL_F32, false, 4, 1>(a, e, s); break;
        case 404: launch_k_hop<WL_F32, false, 4, 4>(a, e, s); break;
        default:
            switch (v / 100) {
            case 1: launch_k_hop<WL_F32, false, 1, 1>(a, e, s); break;
            case 2: launch_k_hop<WL_F32, false, 2, 1>(a, e, s); break;
            case 4: launch_k_hop<WL_F32, false, 4, 1>(a, e, s); break;
            default: launch_k_hop<WL_F32, false, 1, 1>(a, e, s); break;
            }
        }
    }
    WL_CUDA_TRY(cudaGetLastError());
    return WL_OK;
}

template <>
int hop_reduce_launch_prec<WL_F32>(int kind, int dagger, const HopArgs &a, const void *epi, cudaStream_t s)
{
    switch (kind) {
    case 0: launch_reduce_kind<WL_F32, 0>(dagger, a, epi, s); break;
    case 1: launch_reduce_kind<WL_F32, 1>(dagger, a, epi, s); break;
    case 2: launch_reduce_kind<WL_F32, 2>(dagger, a, epi, s); break;
    default: launch_reduce_kind<WL_F32, 3>(dagger, a, epi, s); break;
    }
    WL_CUDA_TRY(cudaGetLastError());
    return WL_OK;
}

}  // namespace wl
