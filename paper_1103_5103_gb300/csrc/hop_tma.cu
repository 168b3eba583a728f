// Wilson hop D_eo / D_oe (Section 2, Eq. 4) with tiles of links and
// neighbour spinors staged in shared memory by the Tensor Memory Accelerator
// (cp.async.bulk.tensor, completion counted on an mbarrier).  Section 4 of
// the paper weighs a shared-memory tile per thread block against one site
// per thread and sets it aside for the hardware of its day; on sm_103a the
// copy engine moves whole boxes of a 5-D tensor view without registers or
// per-thread address arithmetic.
//
// Tile: TY consecutive rows (y) of the Xh sites of one (z, t) slice of the
// output parity, for R right-hand sides; one thread per (site, rhs).  Each
// tile stages, by one elected thread, in one of two stages (the next tile is
// in flight while the current one is computed):
//   - the forward links U_mu(n) of the tile's sites, four directions;
//   - the backward links U_mu(n - mu): x at the tile's rows, y at the rows
//     one below (the row under the tile from a one-row box at the wrapped
//     coordinate), z and t at the tile's rows of the neighbouring slices;
//   - the input spinors of the tile's rows (the x neighbours, and the y
//     neighbours inside the tile) and of the rows just below and above the
//     tile (wrapped), for the R rhs; FP16 with their per-site norms.
// The z and t neighbour spinors, each read by one site of the tile, come
// from global memory directly.
//
// Views of the internal layouts as tensors (innermost first, 4-byte words):
//   spinor  (4 Xh, Y, Z*T, chunk, rhs)   chunk = 16 bytes of one site
//   norms   (Xh, Y, Z*T, rhs)            FP16 only
//   links   (w Xh, Y, Z*T, 3, 4)         the 3 chunks of rows 0-1 of each of 4 directions,
//                                         w = 4 (FP32) or 2 (FP16); row 2 is rebuilt
// Every box starts at x = 0 and spans whole rows, so each copy starts on a
// 16-byte boundary.
//
// Every wait on an mbarrier is bounded (about a second of clock cycles);
// a block that gives up records it in a device word (wl_wait_faults), waits
// (bounded) for its own copy still in flight and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>

#include "hop.cuh"

namespace wl {

__device__ unsigned int g_wait_faults = 0;

namespace {

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity to complete; false after about
// 2^31 clock cycles (about a second at 2 GHz) without completion.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > (1ll << 31)) return false;
    return true;
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int c0, int c1, int c2,
                                            int c3)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6}], [%2];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
        : "memory");
}

__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int c0, int c1, int c2,
                                            int c3, int c4)
{
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6, %7}], "
        "[%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4)
        : "memory");
}

}  // namespace

struct TmaMaps {
    CUtensorMap sp_rows;  // input spinors, box (4 Xh, TY, 1, C, R)
    CUtensorMap sp_row1;  // input spinors, box (4 Xh, 1, 1, C, R)
    CUtensorMap nm_rows;  // FP16 norms, box (Xh, TY, 1, R)
    CUtensorMap nm_row1;  // FP16 norms, box (Xh, 1, 1, R)
    CUtensorMap lk_out;   // output-parity links, box (w Xh, TY, 1, 3, 4)
    CUtensorMap lk_in;    // input-parity links, box (w Xh, TY, 1, 3, 1)
    CUtensorMap lk_in1;   // input-parity links, box (w Xh, 1, 1, 3, 1)
};

// Byte offsets of the regions of one stage.
struct TmaLayout {
    int TY, nyb, ngroups, ntiles;
    int lo, li0, li1a, li1b, li2, li3, spc, spm, spp, nmc, nmm, nmp;
    int stage_bytes;
    unsigned tx_bytes;
};

template <int P> struct TmaIO;

template <> struct TmaIO<WL_F32> {
    static constexpr int C = 6, CB = 16, W = 4;
    // link at (row, xh) of a region [3 or 12 chunks][rows][Xh], chunks ch0..ch0+2
    static __device__ __forceinline__ void link(const unsigned char *reg, int rows, int Xh, int row, int xh, int ch0,
                                                cx<float> (&u)[9])
    {
        const float4 *p = reinterpret_cast<const float4 *>(reg);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float4 t = p[((ch0 + k) * rows + row) * Xh + xh];
            u[2 * k] = {t.x, t.y};
            u[2 * k + 1] = {t.z, t.w};
        }
        reconstruct_row2(u);
    }
    // spinor of rhs rr at (row, xh) of a region [R][C][rows][Xh]; returns the scale
    static __device__ __forceinline__ float spinor(const unsigned char *reg, const unsigned char *, int rows, int Xh,
                                                   int rr, int row, int xh, cx<float> (&v)[12])
    {
        const float4 *p = reinterpret_cast<const float4 *>(reg);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float4 t = p[((rr * 6 + k) * rows + row) * Xh + xh];
            v[2 * k] = {t.x, t.y};
            v[2 * k + 1] = {t.z, t.w};
        }
        return 1.f;
    }
};

template <> struct TmaIO<WL_F16> {
    static constexpr int C = 3, CB = 8, W = 2;
    static __device__ __forceinline__ void link(const unsigned char *reg, int rows, int Xh, int row, int xh, int ch0,
                                                cx<float> (&u)[9])
    {
        const uint2 *p = reinterpret_cast<const uint2 *>(reg);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const uint2 t = p[((ch0 + k) * rows + row) * Xh + xh];
            const float2 a = unpack_half2(t.x), b = unpack_half2(t.y);
            u[2 * k] = {a.x, a.y};
            u[2 * k + 1] = {b.x, b.y};
        }
        reconstruct_row2(u);
    }
    // the norm region is [R][rows][Xh] floats
    static __device__ __forceinline__ float spinor(const unsigned char *reg, const unsigned char *nreg, int rows, int Xh,
                                                   int rr, int row, int xh, cx<float> (&v)[12])
    {
        const uint4 *p = reinterpret_cast<const uint4 *>(reg);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const uint4 t = p[((rr * 3 + k) * rows + row) * Xh + xh];
            const float2 a = unpack_half2(t.x), b = unpack_half2(t.y), c = unpack_half2(t.z), d = unpack_half2(t.w);
            v[4 * k + 0] = {a.x, a.y};
            v[4 * k + 1] = {b.x, b.y};
            v[4 * k + 2] = {c.x, c.y};
            v[4 * k + 3] = {d.x, d.y};
        }
        return reinterpret_cast<const float *>(nreg)[(rr * rows + row) * Xh + xh];
    }
};

// Tile -> (rhs group, row block, z*t slice); rhs groups fastest, so the
// blocks working at one time share links and spinor rows in L2.
struct TileCoord {
    int grp, y0, zt;
};

__device__ __forceinline__ TileCoord tile_coord(const TmaLayout &L, int tile)
{
    TileCoord c;
    c.grp = tile % L.ngroups;
    const int rest = tile / L.ngroups;
    c.y0 = (rest % L.nyb) * L.TY;
    c.zt = rest / L.nyb;
    return c;
}

// Issue the copies of one tile into the stage at st (one thread).
template <int P, int R>
__device__ __forceinline__ void issue_tile(const TmaMaps &m, const TmaLayout &L, const Geom &g, int tile,
                                          unsigned char *st, uint32_t bar)
{
    const TileCoord c = tile_coord(L, tile);
    const int z = c.zt % g.Z, t = c.zt / g.Z;
    const int ym = c.y0 == 0 ? g.Y - 1 : c.y0 - 1;
    const int yp = c.y0 + L.TY == g.Y ? 0 : c.y0 + L.TY;
    const int zm = (z == 0 ? g.Z - 1 : z - 1) + g.Z * t;
    const int tm = z + g.Z * (t == 0 ? g.T - 1 : t - 1);
    const int r0 = c.grp * R;
    mbar_expect_tx(bar, L.tx_bytes);
    tma_load_5d(smem_addr(st + L.lo), &m.lk_out, bar, 0, c.y0, c.zt, 0, 0);
    tma_load_5d(smem_addr(st + L.li0), &m.lk_in, bar, 0, c.y0, c.zt, 0, 0);
    tma_load_5d(smem_addr(st + L.li1a), &m.lk_in1, bar, 0, ym, c.zt, 0, 1);
    tma_load_5d(smem_addr(st + L.li1b), &m.lk_in, bar, 0, c.y0, c.zt, 0, 1);
    tma_load_5d(smem_addr(st + L.li2), &m.lk_in, bar, 0, c.y0, zm, 0, 2);
    tma_load_5d(smem_addr(st + L.li3), &m.lk_in, bar, 0, c.y0, tm, 0, 3);
    tma_load_5d(smem_addr(st + L.spc), &m.sp_rows, bar, 0, c.y0, c.zt, 0, r0);
    tma_load_5d(smem_addr(st + L.spm), &m.sp_row1, bar, 0, ym, c.zt, 0, r0);
    tma_load_5d(smem_addr(st + L.spp), &m.sp_row1, bar, 0, yp, c.zt, 0, r0);
    if constexpr (P == WL_F16) {
        tma_load_4d(smem_addr(st + L.nmc), &m.nm_rows, bar, 0, c.y0, c.zt, r0);
        tma_load_4d(smem_addr(st + L.nmm), &m.nm_row1, bar, 0, ym, c.zt, r0);
        tma_load_4d(smem_addr(st + L.nmp), &m.nm_row1, bar, 0, yp, c.zt, r0);
    }
}

// NREG: the register budget of a thread (128 or 96, no spills): fewer registers,
// more resident warps to hide the global loads of the z and t neighbours.
template <int P, bool DAG, int R, int NREG>
__global__ void __maxnreg__(NREG) k_hop_tma(const __grid_constant__ TmaMaps maps, const TmaLayout L, HopArgs a,
                                             EpiStore epi)
{
    using IO = TmaIO<P>;
    extern __shared__ __align__(128) unsigned char smem[];
    const Geom &g = a.g;
    const int S = L.TY * g.Xh;
    const int tid = threadIdx.x;
    const int s = tid % S, rr = tid / S;
    const int row = s / g.Xh, xh = s % g.Xh;
    const uint32_t bar0 = smem_addr(smem + 2 * L.stage_bytes);
    if (tid == 0) {
        mbar_init(bar0, 1);
        mbar_init(bar0 + 8, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0 && (int)blockIdx.x < L.ntiles) issue_tile<P, R>(maps, L, g, blockIdx.x, smem, bar0);
    int k = 0;
    for (int tile = blockIdx.x; tile < L.ntiles; tile += gridDim.x, ++k) {
        const int stg = k & 1;
        const int next = tile + gridDim.x;
        if (tid == 0 && next < L.ntiles) {
            // the other stage was last read in the previous iteration, which
            // every thread has left (the barrier at its end); order those
            // generic-proxy reads before the copy engine's writes
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue_tile<P, R>(maps, L, g, next, smem + (stg ^ 1) * L.stage_bytes, bar0 + 8 * (stg ^ 1));
        }
        const bool arrived = mbar_wait(bar0 + 8 * stg, (k >> 1) & 1);
        if (__syncthreads_or(!arrived)) {
            if (tid == 0) {
                atomicAdd(&g_wait_faults, 1u);
                // the copy issued for the next tile must land before the
                // block's shared memory is released
                if (next < L.ntiles) mbar_wait(bar0 + 8 * (stg ^ 1), ((k + 1) >> 1) & 1);
            }
            return;
        }
        const unsigned char *st = smem + stg * L.stage_bytes;
        const TileCoord c = tile_coord(L, tile);
        const int r = c.grp * R + rr;
        if (rr < R && r < a.nrhs && !rhs_done(a, r)) {
            const int z = c.zt % g.Z, t = c.zt / g.Z;
            const int y = c.y0 + row;
            const int i = xh + g.Xh * (y + g.Y * c.zt);
            const int x = 2 * xh + ((a.out_parity + y + z + t) & 1);
            const int xf = (x + 1 == g.X ? 0 : x + 1) >> 1, xb = (x == 0 ? g.X - 1 : x - 1) >> 1;
            const int sy = g.Xh * g.Y;
            const int izp = xh + g.Xh * y + sy * ((z + 1 == g.Z ? 0 : z + 1) + g.Z * t);
            const int izm = xh + g.Xh * y + sy * ((z == 0 ? g.Z - 1 : z - 1) + g.Z * t);
            const int itp = xh + g.Xh * y + sy * (z + g.Z * (t + 1 == g.T ? 0 : t + 1));
            const int itm = xh + g.Xh * y + sy * (z + g.Z * (t == 0 ? g.T - 1 : t - 1));
            const bool sf = g.antiperiodic && t + 1 == g.T, sb = g.antiperiodic && t == 0;
            const void *in = static_cast<const char *>(a.in) + (size_t)r * a.rhs_bytes;
            cx<float> acc[1][12];
#pragma unroll
            for (int q = 0; q < 12; ++q) acc[0][q] = acc_zero<float>();
            cx<float> u[9], psi[12];
            float n;
            // x: forward neighbour and link in the tile's rows
            IO::link(st + L.lo, L.TY, g.Xh, row, xh, 0, u);
            n = IO::spinor(st + L.spc, st + L.nmc, L.TY, g.Xh, rr, row, xf, psi);
            transport<0, DAG ? 1 : 0, false>(acc[0], psi, u, n);
            IO::link(st + L.li0, L.TY, g.Xh, row, xb, 0, u);
            n = IO::spinor(st + L.spc, st + L.nmc, L.TY, g.Xh, rr, row, xb, psi);
            transport<0, DAG ? 0 : 1, true>(acc[0], psi, u, n);
            // y: rows above and below, across the tile edge from the halo rows
            IO::link(st + L.lo, L.TY, g.Xh, row, xh, 3, u);
            n = row + 1 < L.TY ? IO::spinor(st + L.spc, st + L.nmc, L.TY, g.Xh, rr, row + 1, xh, psi)
                               : IO::spinor(st + L.spp, st + L.nmp, 1, g.Xh, rr, 0, xh, psi);
            transport<1, DAG ? 1 : 0, false>(acc[0], psi, u, n);
            if (row > 0) {
                IO::link(st + L.li1b, L.TY, g.Xh, row - 1, xh, 0, u);
                n = IO::spinor(st + L.spc, st + L.nmc, L.TY, g.Xh, rr, row - 1, xh, psi);
            } else {
                IO::link(st + L.li1a, 1, g.Xh, 0, xh, 0, u);
                n = IO::spinor(st + L.spm, st + L.nmm, 1, g.Xh, rr, 0, xh, psi);
            }
            transport<1, DAG ? 0 : 1, true>(acc[0], psi, u, n);
            // z: staged links, neighbour spinors from global memory
            IO::link(st + L.lo, L.TY, g.Xh, row, xh, 6, u);
            n = SpinorIO<P>::load_unscaled(in, g.stride, izp, psi);
            transport<2, DAG ? 1 : 0, false>(acc[0], psi, u, n);
            IO::link(st + L.li2, L.TY, g.Xh, row, xh, 0, u);
            n = SpinorIO<P>::load_unscaled(in, g.stride, izm, psi);
            transport<2, DAG ? 0 : 1, true>(acc[0], psi, u, n);
            // t, with the time-boundary sign
            IO::link(st + L.lo, L.TY, g.Xh, row, xh, 9, u);
            n = SpinorIO<P>::load_unscaled(in, g.stride, itp, psi);
            transport<3, DAG ? 1 : 0, false>(acc[0], psi, u, sf ? -n : n);
            IO::link(st + L.li3, L.TY, g.Xh, row, xh, 0, u);
            n = SpinorIO<P>::load_unscaled(in, g.stride, itm, psi);
            transport<3, DAG ? 0 : 1, true>(acc[0], psi, u, sb ? -n : n);
            epi.template operator()<P, 1>(a, i, true, r, acc);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ host

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

int encode(CUtensorMap *m, const void *base, int rank, const cuuint64_t *dims, const cuuint64_t *strides,
           const cuuint32_t *box)
{
    auto fn = encode_fn();
    if (!fn) {
        set_error("TMA hop: cuTensorMapEncodeTiled is not available");
        return WL_ERR_CUDA;
    }
    const cuuint32_t es[5] = {1, 1, 1, 1, 1};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT32, (cuuint32_t)rank, const_cast<void *>(base), dims, strides,
                          box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("TMA hop: cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
        return WL_ERR_CUDA;
    }
    return WL_OK;
}

int align128(int b) { return (b + 127) & ~127; }

template <int P, bool DAG, int R, int NREG>
int launch(const HopArgs &a, const EpiStore &e, cudaStream_t s)
{
    using IO = TmaIO<P>;
    const Geom &g = a.g;
    TmaLayout L;
    L.TY = g.Y % 4 == 0 ? 4 : 2;
    const int threads = L.TY * g.Xh * R;
    // boxes of whole rows: 4 Xh words <= 256; FP16 norm rows of Xh floats and
    // FP16 link rows of 2 Xh words must be multiples of 16 bytes
    if (g.Xh % 4 != 0 || 4 * g.Xh > 256 || threads > 512 || g.Y < L.TY) return WL_VARIANT_NA;
    L.nyb = g.Y / L.TY;
    L.ngroups = (a.nrhs + R - 1) / R;
    const long long ntiles = (long long)L.ngroups * L.nyb * g.Z * g.T;
    if (ntiles > (1ll << 30)) return WL_VARIANT_NA;
    L.ntiles = (int)ntiles;
    const int link_row = g.Xh * IO::CB;          // one chunk of one row of links
    const int sp_row = g.Xh * 16;                // one chunk of one row of spinor
    int off = 0;
    auto region = [&](int bytes) {
        const int o = off;
        off = align128(off + bytes);
        return o;
    };
    L.lo = region(12 * L.TY * link_row);
    L.li0 = region(3 * L.TY * link_row);
    L.li1a = region(3 * link_row);
    L.li1b = region(3 * L.TY * link_row);
    L.li2 = region(3 * L.TY * link_row);
    L.li3 = region(3 * L.TY * link_row);
    L.spc = region(R * IO::C * L.TY * sp_row);
    L.spm = region(R * IO::C * sp_row);
    L.spp = region(R * IO::C * sp_row);
    unsigned tx = (unsigned)(12 * L.TY + 4 * 3 * L.TY + 3) * link_row + (unsigned)R * IO::C * (L.TY + 2) * sp_row;
    if (P == WL_F16) {
        L.nmc = region(R * L.TY * g.Xh * 4);
        L.nmm = region(R * g.Xh * 4);
        L.nmp = region(R * g.Xh * 4);
        tx += (unsigned)R * (L.TY + 2) * g.Xh * 4;
    } else {
        L.nmc = L.nmm = L.nmp = 0;
    }
    L.stage_bytes = off;
    L.tx_bytes = tx;
    const int smem = 2 * L.stage_bytes + 16;
    if (smem > 227 * 1024) return WL_VARIANT_NA;

    TmaMaps m;
    std::memset(&m, 0, sizeof(m));
    const cuuint64_t zt = (cuuint64_t)g.Z * g.T;
    const size_t chunk_stride = (size_t)g.stride * 16;
    {   // spinors (4 Xh, Y, Z T, C, rhs)
        const cuuint64_t dims[5] = {(cuuint64_t)4 * g.Xh, (cuuint64_t)g.Y, zt, (cuuint64_t)IO::C, (cuuint64_t)a.nrhs};
        const cuuint64_t str[4] = {(cuuint64_t)g.Xh * 16, (cuuint64_t)g.Xh * g.Y * 16, chunk_stride, a.rhs_bytes};
        const cuuint32_t b1[5] = {(cuuint32_t)4 * g.Xh, (cuuint32_t)L.TY, 1, (cuuint32_t)IO::C, (cuuint32_t)R};
        const cuuint32_t b2[5] = {(cuuint32_t)4 * g.Xh, 1, 1, (cuuint32_t)IO::C, (cuuint32_t)R};
        WL_TRY(encode(&m.sp_rows, a.in, 5, dims, str, b1));
        WL_TRY(encode(&m.sp_row1, a.in, 5, dims, str, b2));
    }
    if (P == WL_F16) {  // norms (Xh, Y, Z T, rhs) after the 3 chunks
        const void *nb = static_cast<const char *>(a.in) + 3 * chunk_stride;
        const cuuint64_t dims[4] = {(cuuint64_t)g.Xh, (cuuint64_t)g.Y, zt, (cuuint64_t)a.nrhs};
        const cuuint64_t str[3] = {(cuuint64_t)g.Xh * 4, (cuuint64_t)g.Xh * g.Y * 4, a.rhs_bytes};
        const cuuint32_t b1[4] = {(cuuint32_t)g.Xh, (cuuint32_t)L.TY, 1, (cuuint32_t)R};
        const cuuint32_t b2[4] = {(cuuint32_t)g.Xh, 1, 1, (cuuint32_t)R};
        WL_TRY(encode(&m.nm_rows, nb, 4, dims, str, b1));
        WL_TRY(encode(&m.nm_row1, nb, 4, dims, str, b2));
    }
    {   // links (w Xh, Y, Z T, chunk of rows 0-1, direction)
        const cuuint64_t dims[5] = {(cuuint64_t)IO::W * g.Xh, (cuuint64_t)g.Y, zt, 3, 4};
        const cuuint64_t str[4] = {(cuuint64_t)link_row, (cuuint64_t)link_row * g.Y, (cuuint64_t)g.stride * IO::CB,
                                   (cuuint64_t)link_dir_bytes(P, g.stride)};
        const cuuint32_t bo[5] = {(cuuint32_t)IO::W * g.Xh, (cuuint32_t)L.TY, 1, 3, 4};
        const cuuint32_t bi[5] = {(cuuint32_t)IO::W * g.Xh, (cuuint32_t)L.TY, 1, 3, 1};
        const cuuint32_t b1[5] = {(cuuint32_t)IO::W * g.Xh, 1, 1, 3, 1};
        WL_TRY(encode(&m.lk_out, a.links_out, 5, dims, str, bo));
        WL_TRY(encode(&m.lk_in, a.links_in, 5, dims, str, bi));
        WL_TRY(encode(&m.lk_in1, a.links_in, 5, dims, str, b1));
    }
    auto kern = k_hop_tma<P, DAG, R, NREG>;
    static int attr = 0;   // the dynamic shared memory opt-in, raised as needed
    if (smem > attr) {
        WL_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        attr = smem;
    }
    int per_sm = 0;
    WL_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    if (per_sm < 1) return WL_VARIANT_NA;
    const int grid = (int)std::min<long long>(ntiles, (long long)per_sm * sm_count());
    kern<<<grid, threads, smem, s>>>(m, L, a, e);
    return WL_OK;
}

}  // namespace

// Variants 9000 + 100 b + R: R rhs per tile (1, 2 or 4), register budget
// b = 0: 128, 1: 96 per thread (R = 2, 4).  Returns WL_VARIANT_NA for a lattice
// the tiles do not fit (Xh not a multiple of 4, rows too long).
int hop_launch_tma(int prec, int variant, int dagger, const HopArgs &a, const EpiStore &e, cudaStream_t s)
{
    const int R = variant % 100, budget = (variant - 9000) / 100;
    int st = WL_VARIANT_NA;
#define WL_TMA_CASE(PP, RR, BB, NR)                                                                 \
    if (prec == PP && R == RR && budget == BB)                                                      \
        st = dagger ? launch<PP, true, RR, NR>(a, e, s) : launch<PP, false, RR, NR>(a, e, s);
    WL_TMA_CASE(WL_F32, 1, 0, 128)
    WL_TMA_CASE(WL_F32, 2, 0, 128)
    WL_TMA_CASE(WL_F32, 4, 0, 128)
    WL_TMA_CASE(WL_F32, 2, 1, 96)
    WL_TMA_CASE(WL_F32, 4, 1, 96)
    WL_TMA_CASE(WL_F16, 1, 0, 128)
    WL_TMA_CASE(WL_F16, 2, 0, 128)
    WL_TMA_CASE(WL_F16, 4, 0, 128)
    WL_TMA_CASE(WL_F16, 2, 1, 96)
    WL_TMA_CASE(WL_F16, 4, 1, 96)
#undef WL_TMA_CASE
    if (st == WL_VARIANT_NA) set_error("TMA hop variant does not apply to this lattice (X/2 must be a multiple of 4)");
    return st;
}

int wait_faults(unsigned *count, bool reset, cudaStream_t s)
{
    WL_CUDA_TRY(cudaMemcpyFromSymbolAsync(count, g_wait_faults, sizeof(unsigned), 0, cudaMemcpyDeviceToHost, s));
    WL_CUDA_TRY(cudaStreamSynchronize(s));
    if (reset && *count) {
        const unsigned zero = 0;
        WL_CUDA_TRY(cudaMemcpyToSymbolAsync(g_wait_faults, &zero, sizeof(unsigned), 0, cudaMemcpyHostToDevice, s));
        WL_CUDA_TRY(cudaStreamSynchronize(s));
    }
    return WL_OK;
}

}  // namespace wl

using namespace wl;

extern "C" int wl_wait_faults(unsigned *count, int reset, void *stream)
{
    if (!count) {
        set_error("wl_wait_faults: NULL");
        return WL_ERR_ARG;
    }
    return wait_faults(count, reset != 0, as_stream(stream));
}
