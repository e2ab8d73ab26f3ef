// hr_hop_fam.h -- the variants of the hop kernel.  The plain unrolled kernels
// (0, 7) live in hr_hop.cu with the dispatch; every other family has a
// translation unit of its own so that the families compile in parallel:
//   hr_hop_staged.cu  1 cp.async staged, 6 register prefetch
//   hr_hop_loop.cu    2, 3 generic direction loop (registers / staged),
//                     4, 5 loop over mu with switched projections
//   hr_hop_tile.cu    8, 9 near-direction window bulk-copied into shared memory
//   hr_hop_x2.cu      10-13 fundamental FP64 on packed f32x2 FMAs (registers /
//                     cp.async staged, compiler's registers / 96)
//   hr_hop_half.cu    14, 15 fundamental binary16 with the projection in half2
//                     (compiler's registers / 64); 18, 19 the same, cp.async staged;
//                     22, 23 with register prefetch one / two directions ahead
//   hr_hop_p2.cu      16, 17 fundamental FP32 / binary16, two sites per thread in
//                     the lanes of packed f32x2 FMAs (compiler's registers / 96)
//   hr_hop_chunk.cu   20, 21 fundamental FP32 / binary16, a chunk of 2 / 4
//                     right-hand sides per thread sharing the site's links
// All compute the same operator; the autotuner picks per configuration.
#pragma once

#include "hr_host.h"
#include "hr_hop_dev.cuh"

namespace hr {

enum HopVariant : int {
    kVarSimple = 0,
    kVarStaged = 1,
    kVarLoop = 2,
    kVarLoopStaged = 3,
    kVarSwitch = 4,
    kVarSwitchStaged = 5,
    kVarPrefetch = 6,
    kVarSimpleR96 = 7,
    kVarTile = 8,
    kVarTileR96 = 9,
    kVarPaired = 10,
    kVarPairedStaged = 11,
    kVarPairedR96 = 12,
    kVarPairedStagedR96 = 13,
    kVarHalf = 14,
    kVarHalfR64 = 15,
    kVarPairSites = 16,
    kVarPairSitesR96 = 17,
    kVarHalfStaged = 18,
    kVarHalfStagedR64 = 19,
    kVarRhsChunk2 = 20,
    kVarRhsChunk4 = 21,
    kVarHalfPrefetch = 22,
    kVarHalfPrefetch2 = 23
};
static_assert(kVarHalfPrefetch2 + 1 == kNumHopVariants, "variant list");

// per-thread shared-memory slots of the cp.async staged variants (1, 3, 5, 11, 13)
template <int REP, int PREC> struct Stage {
    static constexpr int NC = RepTraits<REP>::NC;
    static constexpr int NV = SpinorLayout<NC, PREC>::NVEC;
    static constexpr int NQ = QuatSlots<PREC>::n;
    static constexpr int NSLOT = NV + NQ + (PREC == kF16 ? 1 : 0); // 16-byte slots per direction
    static size_t smem_bytes(int block) { return (size_t)2 * NSLOT * block * 16; }
};

// direction K = 2 mu + (0 forward, 1 backward): queue its operands' copies
template <int K, int REP, int PREC>
__device__ __forceinline__ void stage_issue(const HopArgs &a, int i, int rr, const SiteNb &nb, uint4 *buf, int bd)
{
    using S = Stage<REP, PREC>;
    constexpr int MU = K >> 1;
    constexpr bool FWD = (K & 1) == 0;
    const int jn = ((FWD ? nb.fwd[MU] : nb.bwd[MU]) << a.g.lrhs) + rr;
    const int site_link = FWD ? i : nb.bwd[MU];
    const int link_par = FWD ? a.p : 1 - a.p;
    const uint4 *src = (const uint4 *)a.in;
#pragma unroll
    for (int v = 0; v < S::NV; ++v) cp_async16(buf + v * bd, src + vec_index(jn, v, S::NV));
#pragma unroll
    for (int v = 0; v < S::NQ; ++v) {
        const void *q = quat_addr<PREC>(a.gauge, a.g.nblk_g, link_par, MU, site_link, v);
        if constexpr (PREC == kF16) cp_async8(buf + (S::NV + v) * bd, q);
        else cp_async16(buf + (S::NV + v) * bd, q);
    }
    if constexpr (PREC == kF16) {
        const float *nrm = (const float *)((const char *)a.in + SpinorLayout<S::NC, PREC>::data_bytes(a.g.nblk_s));
        cp_async4(buf + (S::NV + S::NQ) * bd, nrm + jn);
    }
}

template <int REP, int PREC> constexpr bool has_staged() { return REP != kRepAdjMat; }

// F<REP, PREC>::run(args...) for a run-time (rep, prec); false if invalid
template <template <int, int> class F, class... A> bool for_config(int rep, int prec, A &&...args)
{
    switch (rep * 3 + prec) {
    case 0: return F<kRepFund, kF64>::run(args...);
    case 1: return F<kRepFund, kF32>::run(args...);
    case 2: return F<kRepFund, kF16>::run(args...);
    case 3: return F<kRepAdj, kF64>::run(args...);
    case 4: return F<kRepAdj, kF32>::run(args...);
    case 5: return F<kRepAdj, kF16>::run(args...);
    case 6: return F<kRepAdjMat, kF64>::run(args...);
    case 7: return F<kRepAdjMat, kF32>::run(args...);
    case 8: return F<kRepAdjMat, kF16>::run(args...);
    }
    return false;
}

// Family launchers: start the kernel of variant c.variant for (rep, prec),
// `grid` blocks of c.block threads, and return true with the launch status in
// st; return false if the family has no kernel for this configuration (the
// caller then launches the plain kernel).
bool launch_hop_staged(hr_ctx *ctx, const Geom &g, int rep, int prec, const HopArgs &a, HopChoice c, int grid,
                       cudaStream_t s, hr_status &st);
bool launch_hop_looped(hr_ctx *ctx, const Geom &g, int rep, int prec, const HopArgs &a, HopChoice c, int grid,
                       cudaStream_t s, hr_status &st);
bool launch_hop_tiled(hr_ctx *ctx, const Geom &g, int rep, int prec, const HopArgs &a, HopChoice c, int grid,
                      cudaStream_t s, hr_status &st);
bool launch_hop_paired(hr_ctx *ctx, const Geom &g, int rep, int prec, const HopArgs &a, HopChoice c, int grid,
                       cudaStream_t s, hr_status &st);
bool launch_hop_half(hr_ctx *ctx, const Geom &g, int rep, int prec, const HopArgs &a, HopChoice c, int grid,
                     cudaStream_t s, hr_status &st);
bool launch_hop_pair_sites(hr_ctx *ctx, const Geom &g, int rep, int prec, const HopArgs &a, HopChoice c, int grid,
                           cudaStream_t s, hr_status &st);
bool launch_hop_chunk(hr_ctx *ctx, const Geom &g, int rep, int prec, const HopArgs &a, HopChoice c, int grid,
                      cudaStream_t s, hr_status &st);
// the paired staged kernel with the clover epilogue (fundamental FP64)
void launch_hop_clover_paired(hr_ctx *ctx, const HopArgs &a, int grid, int block, cudaStream_t s, hr_status &st);
// the kernel of lattices with twisted boundaries (hr_hop_twist.cu): every
// operator mode, clover included, kTwistBlock threads per block
constexpr int kTwistBlock = 128;
void launch_hop_twisted(hr_ctx *ctx, int rep, int prec, const HopArgs &a, cudaStream_t s, hr_status &st);

} // namespace hr
