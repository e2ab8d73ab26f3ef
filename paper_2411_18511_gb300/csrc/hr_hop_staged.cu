// hr_hop_staged.cu -- hop variants that hide the neighbour loads behind the
// previous direction's arithmetic: cp.async into per-thread shared-memory slots
// (1) or a second register set (6).
#include <algorithm>
#include <cstdlib>

#include "hr_hop_fam.h"

using namespace hr;

namespace {

// ---------------------------------------------------------------- staged variant


template <int K, int REP, int PREC, class T, int NC>
__device__ __forceinline__ void stage_compute(const HopArgs &a, const uint4 *buf, int bd, cpx<T> (&acc)[4][NC])
{
    using S = Stage<REP, PREC>;
    constexpr int MU = K >> 1;
    constexpr bool FWD = (K & 1) == 0;
    uint4 w[S::NV];
#pragma unroll
    for (int v = 0; v < S::NV; ++v) w[v] = buf[v * bd];
    float sc = 1.f;
    if constexpr (PREC == kF16) sc = *reinterpret_cast<const float *>(buf + (S::NV + S::NQ) * bd);
    cpx<T> s[4][NC];
    spinor_from_vecs<NC, PREC>(w, sc, s);
    uint4 qv[S::NQ];
#pragma unroll
    for (int v = 0; v < S::NQ; ++v) qv[v] = buf[(S::NV + v) * bd];
    T q[4];
    quat_from_vecs<PREC>(qv, q);
    if constexpr (REP == kRepFund) {
        hop_compute<MU, FWD, REP>(s, q, a.g5_in != 0, acc);
    } else {
        T R[3][3];
        quat_to_adj(q, R);
        hop_compute<MU, FWD, REP>(s, R, a.g5_in != 0, acc);
    }
}

// one pipeline step: queue direction K+1 into the other buffer, wait for K, compute K
template <int K, int REP, int PREC, class T, int NC>
__device__ __forceinline__ void stage_step(const HopArgs &a, int i, int rr, const SiteNb &nb, uint4 *b0, uint4 *b1,
                                           int bd, cpx<T> (&acc)[4][NC])
{
    uint4 *cur = (K & 1) ? b1 : b0;
    uint4 *nxt = (K & 1) ? b0 : b1;
    if constexpr (K < 7) {
        stage_issue<K + 1, REP, PREC>(a, i, rr, nb, nxt, bd);
        cp_async_commit();
        cp_async_wait<1>();
    } else {
        cp_async_wait<0>();
    }
    stage_compute<K, REP, PREC>(a, cur, bd, acc);
}

template <int REP, int PREC>
__global__ void __launch_bounds__(256) k_hop_staged(HopArgs a)
{
    using T = typename PrecTraits<PREC>::T;
    using S = Stage<REP, PREC>;
    constexpr int NC = S::NC;
    extern __shared__ uint4 stage_mem[];
    if ((a.gate && *a.gate == 0.0) || (a.done && *a.done != 0.0)) return;
    const Geom &g = a.g;
    const int nv = g.vh << g.lrhs;
    const int stride = gridDim.x * blockDim.x;
    const int bd = blockDim.x;
    // this thread's slots: [buffer][slot][thread], consecutive threads -> consecutive 16 B
    uint4 *b0 = stage_mem + threadIdx.x;
    uint4 *b1 = stage_mem + S::NSLOT * bd + threadIdx.x;
    const T be = Real<T>::from_coef(a.beta);
    const T bu = a.g5_out ? -be : be;
    const T al = Real<T>::from_coef(a.alpha);
    SqAcc<T> red;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nv; j += stride) {
        const int i = j >> g.lrhs, rr = j & (g.nrhs - 1);
        SiteNb nb;
        site_neighbours(g, i, a.p, nb);
        stage_issue<0, REP, PREC>(a, i, rr, nb, b0, bd);
        cp_async_commit();
        cpx<T> acc[4][NC];
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int c = 0; c < NC; ++c) acc[s][c] = {T(0), T(0)};
        stage_step<0, REP, PREC>(a, i, rr, nb, b0, b1, bd, acc);
        stage_step<1, REP, PREC>(a, i, rr, nb, b0, b1, bd, acc);
        stage_step<2, REP, PREC>(a, i, rr, nb, b0, b1, bd, acc);
        stage_step<3, REP, PREC>(a, i, rr, nb, b0, b1, bd, acc);
        stage_step<4, REP, PREC>(a, i, rr, nb, b0, b1, bd, acc);
        stage_step<5, REP, PREC>(a, i, rr, nb, b0, b1, bd, acc);
        stage_step<6, REP, PREC>(a, i, rr, nb, b0, b1, bd, acc);
        stage_step<7, REP, PREC>(a, i, rr, nb, b0, b1, bd, acc);
        hop_epilogue<PREC>(a, j, acc, al, be, bu, red);
    }
    if (a.fin) {
        __shared__ double smem[32 * 32];
        __shared__ double sums[32];
        if (grid_reduce(red, g.nrhs, a.red, sums, smem)) finish_reduction(a.fin, sums, g.nrhs, a.scal);
    }
}

// ---------------------------------------------------------------- prefetching variant
// Unrolled like k_hop, but the operands of direction k+1 are loaded into a
// second set of registers before direction k is computed, so every load has a
// whole direction of arithmetic to arrive in.  Costs registers (two operand
// sets) and so occupancy; the autotuner decides whether it pays.

template <int K, int REP, int PREC, class T, int NC>
__device__ __forceinline__ void pf_load(const HopArgs &a, int i, int rr, const SiteNb &nb, cpx<T> (&s)[4][NC],
                                        T (&q)[4], float &sc)
{
    constexpr int MU = K >> 1;
    constexpr bool FWD = (K & 1) == 0;
    const int nbr = FWD ? nb.fwd[MU] : nb.bwd[MU];
    load_spinor_raw<NC, PREC>(a.in, a.g.nblk_s, (nbr << a.g.lrhs) + rr, s, sc);
    load_quat<PREC>(a.gauge, a.g.nblk_g, FWD ? a.p : 1 - a.p, MU, FWD ? i : nb.bwd[MU], q);
}

template <int K, int REP, int PREC, class T, int NC>
__device__ __forceinline__ void pf_compute(const HopArgs &a, cpx<T> (&s)[4][NC], T (&q)[4], float sc,
                                           cpx<T> (&acc)[4][NC])
{
    constexpr int MU = K >> 1;
    constexpr bool FWD = (K & 1) == 0;
    if constexpr (REP == kRepFund) {
        if constexpr (PREC == kF16) {
#pragma unroll
            for (int k = 0; k < 4; ++k) q[k] = q[k] * sc;
        }
        hop_compute<MU, FWD, REP>(s, q, a.g5_in != 0, acc);
    } else {
        T R[3][3];
        quat_to_adj(q, R);
        if constexpr (PREC == kF16) {
#pragma unroll
            for (int k = 0; k < 9; ++k) R[k / 3][k % 3] = R[k / 3][k % 3] * sc;
        }
        hop_compute<MU, FWD, REP>(s, R, a.g5_in != 0, acc);
    }
}

template <int REP, int PREC>
__global__ void __launch_bounds__(256) k_hop_pf(HopArgs a)
{
    using T = typename PrecTraits<PREC>::T;
    constexpr int NC = RepTraits<REP>::NC;
    if ((a.gate && *a.gate == 0.0) || (a.done && *a.done != 0.0)) return;
    const Geom &g = a.g;
    const int nv = g.vh << g.lrhs;
    const int stride = gridDim.x * blockDim.x;
    const T be = Real<T>::from_coef(a.beta);
    const T bu = a.g5_out ? -be : be;
    const T al = Real<T>::from_coef(a.alpha);
    SqAcc<T> red;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nv; j += stride) {
        const int i = j >> g.lrhs, rr = j & (g.nrhs - 1);
        SiteNb nb;
        site_neighbours(g, i, a.p, nb);
        cpx<T> acc[4][NC];
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int c = 0; c < NC; ++c) acc[s][c] = {T(0), T(0)};
        cpx<T> sA[4][NC], sB[4][NC];
        T qA[4], qB[4];
        float cA, cB;
        pf_load<0, REP, PREC>(a, i, rr, nb, sA, qA, cA);
        pf_load<1, REP, PREC>(a, i, rr, nb, sB, qB, cB);
        pf_compute<0, REP, PREC>(a, sA, qA, cA, acc);
        pf_load<2, REP, PREC>(a, i, rr, nb, sA, qA, cA);
        pf_compute<1, REP, PREC>(a, sB, qB, cB, acc);
        pf_load<3, REP, PREC>(a, i, rr, nb, sB, qB, cB);
        pf_compute<2, REP, PREC>(a, sA, qA, cA, acc);
        pf_load<4, REP, PREC>(a, i, rr, nb, sA, qA, cA);
        pf_compute<3, REP, PREC>(a, sB, qB, cB, acc);
        pf_load<5, REP, PREC>(a, i, rr, nb, sB, qB, cB);
        pf_compute<4, REP, PREC>(a, sA, qA, cA, acc);
        pf_load<6, REP, PREC>(a, i, rr, nb, sA, qA, cA);
        pf_compute<5, REP, PREC>(a, sB, qB, cB, acc);
        pf_load<7, REP, PREC>(a, i, rr, nb, sB, qB, cB);
        pf_compute<6, REP, PREC>(a, sA, qA, cA, acc);
        pf_compute<7, REP, PREC>(a, sB, qB, cB, acc);
        hop_epilogue<PREC>(a, j, acc, al, be, bu, red);
    }
    if (a.fin) {
        __shared__ double smem[32 * 32];
        __shared__ double sums[32];
        if (grid_reduce(red, g.nrhs, a.red, sums, smem)) finish_reduction(a.fin, sums, g.nrhs, a.scal);
    }
}

template <int REP, int PREC> struct Launch {
    static bool run(hr_ctx *ctx, const Geom &, const HopArgs &a, HopChoice c, int grid, cudaStream_t s,
                    hr_status &st)
    {
        if constexpr (has_staged<REP, PREC>()) {
            if (c.variant == kVarStaged) {
                const size_t sm = Stage<REP, PREC>::smem_bytes(c.block);
                static bool attr_set = false;
                if (!attr_set) {
                    cudaFuncSetAttribute(k_hop_staged<REP, PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Stage<REP, PREC>::smem_bytes(256));
                    attr_set = true;
                }
                k_hop_staged<REP, PREC><<<grid, c.block, sm, s>>>(a);
                st = check_launch(ctx, "staged hop kernel");
                return true;
            }
            if (c.variant == kVarPrefetch) {
                k_hop_pf<REP, PREC><<<grid, c.block, 0, s>>>(a);
                st = check_launch(ctx, "prefetching hop kernel");
                return true;
            }
        }
        return false;
    }
};

} // namespace

namespace hr {

bool launch_hop_staged(hr_ctx *ctx, const Geom &g, int rep, int prec, const HopArgs &a, HopChoice c, int grid,
                       cudaStream_t s, hr_status &st)
{
    return for_config<Launch>(rep, prec, ctx, g, a, c, grid, s, st);
}

} // namespace hr
