// hr_hop_half.cu -- the binary16 fundamental hop with the spin projection in
// half2 arithmetic (variants 14, 15, 18, 19, 22, 23).
//
// The FP16 hop moves 136 bytes per output site (the neighbour spinors as
// binary16 with one FP32 scale per site, binary16 quaternion links), so at
// the HBM copy rate it has about 800 instruction issues per site to spend,
// and the FP32-arithmetic kernels spend more: they widen all 16 stored
// halves of every neighbour to floats before projecting.  Here the
// projection h_t = s_t + i^c s_pi of (1 -/+ g_mu) runs on the stored halves
// themselves -- a packed word holds one part (re or im) of both colours, so a
// half-spinor is four HADD2 -- and only the 8 projected halves are widened.
// The neighbour's scale rides on the rebuild instead of the link: every
// accumulation acc (+)= i^k sc r is one FMA with +-sc as its multiplier.
//
// Precision: the half2 addition rounds the projected components to binary16
// (a relative 2^-11 of the neighbour site's largest component), the same
// size as the storage rounding of the components it adds; the colour product
// and the accumulation run in FP32.  The result agrees with the FP32-
// arithmetic kernels to the storage precision, not bit for bit.
//
// Variant 14: registers as the compiler likes; 15: capped at 64 registers;
// 18, 19: the same with the next direction's operands staged by cp.async;
// 22, 23: with the operands of the next direction (80 registers) or of the
// next two (96 registers) loaded into registers ahead of the arithmetic.
#include "hr_hop_fam.h"
#include "hr_hop_x2.cuh"

using namespace hr;

namespace {

// the neighbour and link loaded from global memory
template <int MU, bool FWD, bool FIRST, bool NEG>
__device__ __forceinline__ void h16_term(const HopArgs &a, const float *nrm, int site_link, int link_par, int jn,
                                         cpx<float> (&acc)[4][2])
{
    const uint4 *sp = (const uint4 *)a.in;
    const uint4 w0 = __ldg(sp + vec_index(jn, 0, 2));
    const uint4 w1 = __ldg(sp + vec_index(jn, 1, 2));
    const float sc = __ldg(nrm + jn);
    float q[4];
    load_quat<kF16>(a.gauge, a.g.nblk_g, link_par, MU, site_link, q);
    h16_compute<MU, FWD, FIRST, NEG>(w0, w1, sc, q, acc);
}

template <int MU, bool FIRST, bool NEG>
__device__ __forceinline__ void h16_dir(const HopArgs &a, const float *nrm, int i, int rr, const SiteNb &nb,
                                        cpx<float> (&acc)[4][2])
{
    const int l = a.g.lrhs;
    h16_term<MU, true, FIRST, NEG>(a, nrm, i, a.p, (nb.fwd[MU] << l) + rr, acc);
    h16_term<MU, false, false, NEG>(a, nrm, nb.bwd[MU], 1 - a.p, (nb.bwd[MU] << l) + rr, acc);
}

template <int G5IN>
__device__ __forceinline__ void h16_body(const HopArgs &a)
{
    constexpr bool NEG = G5IN != 0;
    if ((a.gate && *a.gate == 0.0) || (a.done && *a.done != 0.0)) return;
    const Geom &g = a.g;
    const int nv = g.vh << g.lrhs;
    const int stride = gridDim.x * blockDim.x;
    const float *nrm = (const float *)((const char *)a.in + SpinorLayout<2, kF16>::data_bytes(g.nblk_s));
    const float be = a.beta.h;
    const float bu = a.g5_out ? -be : be;
    const float al = a.alpha.h;
    SqAcc<float> red;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nv; j += stride) {
        const int i = j >> g.lrhs, rr = j & (g.nrhs - 1);
        SiteNb nb;
        site_neighbours(g, i, a.p, nb);
        cpx<float> acc[4][2];
        h16_dir<0, true, NEG>(a, nrm, i, rr, nb, acc);
        h16_dir<1, false, NEG>(a, nrm, i, rr, nb, acc);
        h16_dir<2, false, NEG>(a, nrm, i, rr, nb, acc);
        h16_dir<3, false, NEG>(a, nrm, i, rr, nb, acc);
        hop_epilogue<kF16>(a, j, acc, al, be, bu, red);
    }
    if (a.fin) {
        __shared__ double smem[32 * 32];
        __shared__ double sums[32];
        if (grid_reduce(red, g.nrhs, a.red, sums, smem)) finish_reduction(a.fin, sums, g.nrhs, a.scal);
    }
}

// Register-prefetch form: direction K+1's two spinor words, scale and link
// are loaded into registers before direction K is computed, so each thread
// keeps one direction's loads in flight behind its arithmetic.
struct H16Ops {
    uint4 w0, w1;
    float sc;
    uint2 q;
};

template <int K>
__device__ __forceinline__ void h16_fetch(const HopArgs &a, const float *nrm, int i, int rr, const SiteNb &nb,
                                          H16Ops &o)
{
    constexpr int MU = K >> 1;
    constexpr bool FWD = (K & 1) == 0;
    const int jn = ((FWD ? nb.fwd[MU] : nb.bwd[MU]) << a.g.lrhs) + rr;
    const int sl = FWD ? i : nb.bwd[MU];
    const int lp = FWD ? a.p : 1 - a.p;
    const uint4 *sp = (const uint4 *)a.in;
    o.w0 = __ldg(sp + vec_index(jn, 0, 2));
    o.w1 = __ldg(sp + vec_index(jn, 1, 2));
    o.sc = __ldg(nrm + jn);
    o.q = __ldg((const uint2 *)quat_addr<kF16>(a.gauge, a.g.nblk_g, lp, MU, sl, 0));
}

// direction K from buf[K % (D + 1)] after queueing the loads of direction K + D
template <int K, int D, bool NEG>
__device__ __forceinline__ void h16p_step(const HopArgs &a, const float *nrm, int i, int rr, const SiteNb &nb,
                                          H16Ops (&buf)[D + 1], cpx<float> (&acc)[4][2])
{
    if constexpr (K + D < 8) h16_fetch<K + D>(a, nrm, i, rr, nb, buf[(K + D) % (D + 1)]);
    const H16Ops &cur = buf[K % (D + 1)];
    const float2 q01 = __half22float2(as_h2(cur.q.x)), q23 = __half22float2(as_h2(cur.q.y));
    const float q[4] = {q01.x, q01.y, q23.x, q23.y};
    h16_compute<(K >> 1), (K & 1) == 0, K == 0, NEG>(cur.w0, cur.w1, cur.sc, q, acc);
}

// D: how many directions ahead the loads run (1 or 2)
template <int D, int G5IN>
__device__ __forceinline__ void h16p_body(const HopArgs &a)
{
    constexpr bool NEG = G5IN != 0;
    if ((a.gate && *a.gate == 0.0) || (a.done && *a.done != 0.0)) return;
    const Geom &g = a.g;
    const int nv = g.vh << g.lrhs;
    const int stride = gridDim.x * blockDim.x;
    const float *nrm = (const float *)((const char *)a.in + SpinorLayout<2, kF16>::data_bytes(g.nblk_s));
    const float be = a.beta.h;
    const float bu = a.g5_out ? -be : be;
    const float al = a.alpha.h;
    SqAcc<float> red;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nv; j += stride) {
        const int i = j >> g.lrhs, rr = j & (g.nrhs - 1);
        SiteNb nb;
        site_neighbours(g, i, a.p, nb);
        epilogue_prefetch<2, kF16>(a, j);
        H16Ops buf[D + 1];
        h16_fetch<0>(a, nrm, i, rr, nb, buf[0]);
        if constexpr (D > 1) h16_fetch<1>(a, nrm, i, rr, nb, buf[1]);
        cpx<float> acc[4][2];
        h16p_step<0, D, NEG>(a, nrm, i, rr, nb, buf, acc);
        h16p_step<1, D, NEG>(a, nrm, i, rr, nb, buf, acc);
        h16p_step<2, D, NEG>(a, nrm, i, rr, nb, buf, acc);
        h16p_step<3, D, NEG>(a, nrm, i, rr, nb, buf, acc);
        h16p_step<4, D, NEG>(a, nrm, i, rr, nb, buf, acc);
        h16p_step<5, D, NEG>(a, nrm, i, rr, nb, buf, acc);
        h16p_step<6, D, NEG>(a, nrm, i, rr, nb, buf, acc);
        h16p_step<7, D, NEG>(a, nrm, i, rr, nb, buf, acc);
        hop_epilogue<kF16>(a, j, acc, al, be, bu, red);
    }
    if (a.fin) {
        __shared__ double smem[32 * 32];
        __shared__ double sums[32];
        if (grid_reduce(red, g.nrhs, a.red, sums, smem)) finish_reduction(a.fin, sums, g.nrhs, a.scal);
    }
}

// Staged form: direction K+1's two spinor words, link and scale are copied by
// cp.async into this thread's shared-memory slots while direction K is
// computed from the other buffer, so each warp keeps a direction's operands in
// flight without holding them in registers.
template <int K, bool NEG>
__device__ __forceinline__ void h16_stage_step(const HopArgs &a, int i, int rr, const SiteNb &nb, uint4 *b0,
                                               uint4 *b1, int bd, cpx<float> (&acc)[4][2])
{
    using S = Stage<kRepFund, kF16>;
    static_assert(S::NV == 2 && S::NQ == 1 && S::NSLOT == 4, "two spinor words, the link, the scale");
    uint4 *cur = (K & 1) ? b1 : b0;
    uint4 *nxt = (K & 1) ? b0 : b1;
    if constexpr (K < 7) {
        stage_issue<K + 1, kRepFund, kF16>(a, i, rr, nb, nxt, bd);
        cp_async_commit();
        cp_async_wait<1>();
    } else {
        cp_async_wait<0>();
    }
    const uint4 w0 = cur[0], w1 = cur[bd];
    const uint2 qw = *reinterpret_cast<const uint2 *>(cur + 2 * bd); // the link slot holds 8 bytes
    const float sc = *reinterpret_cast<const float *>(cur + 3 * bd);  // the scale slot 4
    const float2 q01 = __half22float2(as_h2(qw.x)), q23 = __half22float2(as_h2(qw.y));
    const float q[4] = {q01.x, q01.y, q23.x, q23.y};
    h16_compute<(K >> 1), (K & 1) == 0, K == 0, NEG>(w0, w1, sc, q, acc);
}

template <int G5IN>
__device__ __forceinline__ void h16s_body(const HopArgs &a)
{
    using S = Stage<kRepFund, kF16>;
    constexpr bool NEG = G5IN != 0;
    extern __shared__ uint4 h16_stage_mem[];
    if ((a.gate && *a.gate == 0.0) || (a.done && *a.done != 0.0)) return;
    const Geom &g = a.g;
    const int nv = g.vh << g.lrhs;
    const int stride = gridDim.x * blockDim.x;
    const int bd = blockDim.x;
    uint4 *b0 = h16_stage_mem + threadIdx.x;
    uint4 *b1 = h16_stage_mem + S::NSLOT * bd + threadIdx.x;
    const float be = a.beta.h;
    const float bu = a.g5_out ? -be : be;
    const float al = a.alpha.h;
    SqAcc<float> red;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nv; j += stride) {
        const int i = j >> g.lrhs, rr = j & (g.nrhs - 1);
        SiteNb nb;
        site_neighbours(g, i, a.p, nb);
        stage_issue<0, kRepFund, kF16>(a, i, rr, nb, b0, bd);
        cp_async_commit();
        cpx<float> acc[4][2];
        h16_stage_step<0, NEG>(a, i, rr, nb, b0, b1, bd, acc);
        h16_stage_step<1, NEG>(a, i, rr, nb, b0, b1, bd, acc);
        h16_stage_step<2, NEG>(a, i, rr, nb, b0, b1, bd, acc);
        h16_stage_step<3, NEG>(a, i, rr, nb, b0, b1, bd, acc);
        h16_stage_step<4, NEG>(a, i, rr, nb, b0, b1, bd, acc);
        h16_stage_step<5, NEG>(a, i, rr, nb, b0, b1, bd, acc);
        h16_stage_step<6, NEG>(a, i, rr, nb, b0, b1, bd, acc);
        h16_stage_step<7, NEG>(a, i, rr, nb, b0, b1, bd, acc);
        hop_epilogue<kF16>(a, j, acc, al, be, bu, red);
    }
    if (a.fin) {
        __shared__ double smem[32 * 32];
        __shared__ double sums[32];
        if (grid_reduce(red, g.nrhs, a.red, sums, smem)) finish_reduction(a.fin, sums, g.nrhs, a.scal);
    }
}

template <int G5IN> __global__ void __launch_bounds__(256) k_hop_h16(HopArgs a) { h16_body<G5IN>(a); }
template <int G5IN> __global__ void __maxnreg__(64) k_hop_h16_r64(HopArgs a) { h16_body<G5IN>(a); }
template <int G5IN> __global__ void __launch_bounds__(256) k_hop_h16s(HopArgs a) { h16s_body<G5IN>(a); }
template <int G5IN> __global__ void __maxnreg__(64) k_hop_h16s_r64(HopArgs a) { h16s_body<G5IN>(a); }
template <int G5IN> __global__ void __maxnreg__(80) k_hop_h16p_r80(HopArgs a) { h16p_body<1, G5IN>(a); }
template <int G5IN> __global__ void __maxnreg__(96) k_hop_h16p2_r96(HopArgs a) { h16p_body<2, G5IN>(a); }

} // namespace

namespace hr {

bool launch_hop_half(hr_ctx *ctx, const Geom &, int rep, int prec, const HopArgs &a, HopChoice c, int grid,
                     cudaStream_t s, hr_status &st)
{
    if (rep != HR_FUND || prec != kF16) return false;
    const bool g5 = a.g5_in != 0;
    if (c.variant == kVarHalfStaged || c.variant == kVarHalfStagedR64) {
        using S = Stage<kRepFund, kF16>;
        static bool attr_set = false;
        if (!attr_set) {
            for (auto f : {k_hop_h16s<0>, k_hop_h16s<1>, k_hop_h16s_r64<0>, k_hop_h16s_r64<1>})
                cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::smem_bytes(256));
            attr_set = true;
        }
        const size_t sm = S::smem_bytes(c.block);
        if (c.variant == kVarHalfStagedR64) (g5 ? k_hop_h16s_r64<1> : k_hop_h16s_r64<0>)<<<grid, c.block, sm, s>>>(a);
        else (g5 ? k_hop_h16s<1> : k_hop_h16s<0>)<<<grid, c.block, sm, s>>>(a);
    } else if (c.variant == kVarHalfR64) {
        (g5 ? k_hop_h16_r64<1> : k_hop_h16_r64<0>)<<<grid, c.block, 0, s>>>(a);
    } else if (c.variant == kVarHalfPrefetch) {
        (g5 ? k_hop_h16p_r80<1> : k_hop_h16p_r80<0>)<<<grid, c.block, 0, s>>>(a);
    } else if (c.variant == kVarHalfPrefetch2) {
        (g5 ? k_hop_h16p2_r96<1> : k_hop_h16p2_r96<0>)<<<grid, c.block, 0, s>>>(a);
    } else {
        (g5 ? k_hop_h16<1> : k_hop_h16<0>)<<<grid, c.block, 0, s>>>(a);
    }
    st = check_launch(ctx, "binary16 hop kernel (half2 projection)");
    return true;
}

} // namespace hr
