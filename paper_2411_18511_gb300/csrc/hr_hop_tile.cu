// hr_hop_tile.cu -- the tiled hop (variants 8, 9): the near-direction
// neighbours of a tile come from a window of the input bulk-copied (TMA) into
// shared memory.
#include <algorithm>
#include <cstdlib>

#include "hr_hop_fam.h"

using namespace hr;

namespace {

// ---------------------------------------------------------------- tiled variant
// A tile is blockDim.x consecutive output (virtual) sites.  Their neighbours in
// the two fastest directions -- mu = 3 inside the row, mu = 2 one row (h3
// sites) away -- lie within h3 sites of the tile except across the periodic
// wrap of those directions.  In the AoSoA layout that window of the input field
// is one contiguous run of 32-site blocks, so one thread queues it as a single
// bulk (TMA) copy into shared memory when the tile starts.  The block works on
// the far directions mu = 0, 1 from global memory meanwhile, then takes mu = 2,
// 3 from shared memory (a wrapping neighbour from global memory): half of the
// neighbour spinors no longer wait on L2.

template <int REP, int PREC> struct TileStage {
    static constexpr int NC = RepTraits<REP>::NC;
    static constexpr int NV = SpinorLayout<NC, PREC>::NVEC;
    static constexpr size_t kBlockBytes = (size_t)NV * 32 * 16; // one 32-site AoSoA block
    static constexpr size_t kHead = 128;                        // mbarrier, then the stage
    // the window [i_lo - h3, i_hi + h3] of a tile of `block` virtual sites spans
    // at most block + (2 h3 + 1) nrhs virtual sites, plus a partial block at each end
    static int max_blocks(const Geom &g, int block) { return (block + (2 * g.h3 + 1) * g.nrhs) / 32 + 3; }
    static size_t smem_bytes(const Geom &g, int block) { return kHead + (size_t)max_blocks(g, block) * kBlockBytes; }
};
constexpr size_t kTileSmemMax = 100 * 1024; // larger windows use the plain kernel

template <int MU, bool FWD, int REP, int PREC, class T, int NC>
__device__ __forceinline__ void tile_term(const HopArgs &a, int site_link, int link_par, int j_nb, bool neg_upper,
                                          const uint4 *stage, int js_lo, int js_hi, bool landed, cpx<T> (&acc)[4][NC])
{
    constexpr int NV = SpinorLayout<NC, PREC>::NVEC;
    // one load sequence through a generic pointer, into the window or into the
    // field: no second copy of the load code for the wrapping neighbours
    const bool staged = landed && j_nb >= js_lo && j_nb < js_hi;
    const int jj = staged ? j_nb - js_lo : j_nb;
    const uint4 *p = (staged ? stage : (const uint4 *)a.in) + (size_t)(jj >> 5) * NV * 32 + (jj & 31);
    uint4 w[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) w[v] = p[v * 32];
    cpx<T> s[4][NC];
    spinor_from_vecs<NC, PREC>(w, 1.f, s);
    hop_term_with<MU, FWD, REP, PREC>(a, site_link, link_par, s, 1.f, neg_upper, acc);
}

template <int REP, int PREC, int G5IN>
__device__ __forceinline__ void hop_tile_body(const HopArgs &a)
{
    using T = typename PrecTraits<PREC>::T;
    using S = TileStage<REP, PREC>;
    constexpr int NC = S::NC, NV = S::NV;
    static_assert(PREC != kF16, "binary16 sites carry a separate scale array");
    extern __shared__ __align__(128) unsigned char tile_smem[];
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(tile_smem);
    const uint4 *stage = reinterpret_cast<const uint4 *>(tile_smem + S::kHead);
    __shared__ int s_landed;
    if ((a.gate && *a.gate == 0.0) || (a.done && *a.done != 0.0)) return;
    const Geom &g = a.g;
    const int l = g.lrhs;
    const int nv = g.vh << l;
    const int ntiles = (nv + blockDim.x - 1) / blockDim.x;
    const T be = Real<T>::from_coef(a.beta);
    const T bu = a.g5_out ? -be : be;
    const T al = Real<T>::from_coef(a.alpha);
    const bool neg = g5_in_of<G5IN>(a);
    SqAcc<T> red;
    unsigned dyn_smem;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn_smem));
    if (threadIdx.x == 0) mbar_init(bar, 1);
    __syncthreads();
    unsigned phase = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int j0 = tile * blockDim.x;
        const int jend = min(j0 + (int)blockDim.x, nv);
        const int i_lo = j0 >> l, i_hi = (jend - 1) >> l;
        const int v_lo = max(0, i_lo - g.h3) << l;
        const int v_hi = min(g.vh, i_hi + g.h3 + 1) << l;
        const int b_lo = v_lo >> 5, b_hi = (v_hi + 31) >> 5; // b_hi <= nblk_s
        const int js_lo = b_lo << 5, js_hi = b_hi << 5;
        // block-uniform: the window fits the shared memory this launch was given
        const bool use_stage = S::kHead + (size_t)(b_hi - b_lo) * S::kBlockBytes <= dyn_smem;
        if (use_stage && threadIdx.x == 0) {
            // the block's reads of the previous window are ordered before this copy
            fence_proxy_async_smem();
            const unsigned bytes = (unsigned)((size_t)(b_hi - b_lo) * S::kBlockBytes);
            if (a.inject_no_copy) mbar_arrive_expect_tx(bar, bytes); // test: the copy never comes
            else bulk_copy_g2s(tile_smem + S::kHead, (const uint4 *)a.in + (size_t)b_lo * NV * 32, bytes, bar);
        }
        const int j = j0 + threadIdx.x;
        const bool act = j < nv;
        cpx<T> acc[4][NC];
        SiteNb nb;
        int i = 0, rr = 0;
        if (act) {
            i = j >> l;
            rr = j & (g.nrhs - 1);
            site_neighbours(g, i, a.p, nb);
            hop_dir<0, REP, PREC, G5IN, true>(a, i, rr, nb, acc);
            hop_dir<1, REP, PREC, G5IN>(a, i, rr, nb, acc);
        }
        // a copy that has not landed after about a second: take every neighbour
        // from global memory (same result) and let the block vote below
        const bool landed = use_stage && mbar_wait_bounded(bar, phase, a.wait_cycles);
        if (act) {
            tile_term<2, true, REP, PREC>(a, i, a.p, (nb.fwd[2] << l) + rr, neg, stage, js_lo, js_hi, landed, acc);
            tile_term<2, false, REP, PREC>(a, nb.bwd[2], 1 - a.p, (nb.bwd[2] << l) + rr, neg, stage, js_lo, js_hi,
                                           landed, acc);
            tile_term<3, true, REP, PREC>(a, i, a.p, (nb.fwd[3] << l) + rr, neg, stage, js_lo, js_hi, landed, acc);
            tile_term<3, false, REP, PREC>(a, nb.bwd[3], 1 - a.p, (nb.bwd[3] << l) + rr, neg, stage, js_lo, js_hi,
                                           landed, acc);
            hop_epilogue<PREC>(a, j, acc, al, be, bu, red);
        }
        // end of the tile: nobody reads the window any more; if a copy timed
        // out, wait for it once more before the buffer is refilled or the block
        // exits, and give up (recording a device error) if it still has not landed
        if (!use_stage) continue; // no copy queued, the barrier phase stays
        if (tile + (int)gridDim.x >= ntiles) {
            // the block's last tile: a thread that saw the copy land may leave;
            // one that did not waits once more before the block can exit
            if (!landed && !mbar_wait_bounded(bar, phase, a.wait_cycles) && a.scal)
                sc(a.scal, S_FLAGS, F_DEVERR) = 1.0;
            break;
        }
        if (__syncthreads_or(!landed)) {
            if (threadIdx.x == 0) {
                s_landed = mbar_wait_bounded(bar, phase, a.wait_cycles) ? 1 : 0;
                if (a.scal) sc(a.scal, S_FLAGS, F_DEVERR) = 1.0;
            }
            __syncthreads();
            if (!s_landed) break;
        }
        phase ^= 1u;
    }
    if (a.fin) {
        __shared__ double smem[32 * 32];
        __shared__ double sums[32];
        if (grid_reduce(red, g.nrhs, a.red, sums, smem)) finish_reduction(a.fin, sums, g.nrhs, a.scal);
    }
}

template <int REP, int PREC, int G5IN>
__global__ void __launch_bounds__(256) k_hop_tile(HopArgs a)
{
    hop_tile_body<REP, PREC, G5IN>(a);
}

template <int REP, int PREC, int G5IN>
__global__ void __maxnreg__(96) k_hop_tile_r96(HopArgs a)
{
    hop_tile_body<REP, PREC, G5IN>(a);
}

template <int REP, int PREC> struct Launch {
    static bool run(hr_ctx *ctx, const Geom &g, const HopArgs &a, HopChoice c, int, cudaStream_t s, hr_status &st)
    {
        if constexpr (PREC != kF16) {
            using S = TileStage<REP, PREC>;
            const size_t sm = S::smem_bytes(g, c.block);
            if (sm > kTileSmemMax) return false; // the window does not fit: plain kernel
            static bool attr_tile = false;
            if (!attr_tile) {
                cudaFuncSetAttribute(k_hop_tile<REP, PREC, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kTileSmemMax);
                cudaFuncSetAttribute(k_hop_tile<REP, PREC, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kTileSmemMax);
                cudaFuncSetAttribute(k_hop_tile_r96<REP, PREC, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kTileSmemMax);
                cudaFuncSetAttribute(k_hop_tile_r96<REP, PREC, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kTileSmemMax);
                attr_tile = true;
            }
            // one tile per block; a reducing launch loops over tiles within the partials' cap
            const long long nv = (long long)g.vh << g.lrhs;
            const long long ntiles = (nv + c.block - 1) / c.block;
            const int tgrid = (int)std::min<long long>(ntiles, a.fin ? kMaxBlocks : (1LL << 30));
            if (c.variant == kVarTile) {
                if (a.g5_in) k_hop_tile<REP, PREC, 1><<<tgrid, c.block, sm, s>>>(a);
                else k_hop_tile<REP, PREC, 0><<<tgrid, c.block, sm, s>>>(a);
            } else {
                if (a.g5_in) k_hop_tile_r96<REP, PREC, 1><<<tgrid, c.block, sm, s>>>(a);
                else k_hop_tile_r96<REP, PREC, 0><<<tgrid, c.block, sm, s>>>(a);
            }
            st = check_launch(ctx, "tiled hop kernel");
            return true;
        }
        return false;
    }
};

} // namespace

namespace hr {

bool launch_hop_tiled(hr_ctx *ctx, const Geom &g, int rep, int prec, const HopArgs &a, HopChoice c, int grid,
                      cudaStream_t s, hr_status &st)
{
    return for_config<Launch>(rep, prec, ctx, g, a, c, grid, s, st);
}

} // namespace hr
