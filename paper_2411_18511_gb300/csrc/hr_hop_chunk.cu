// hr_hop_chunk.cu -- the fundamental FP32 / binary16 hop with a chunk of C
// right-hand sides per thread (variants 20: C = 2, 21: C = 4).
//
// With N right-hand sides the layout puts the N virtual sites j = i N + r of a
// lattice site next to each other, and the one-RHS-per-thread kernels give each
// of them a thread: every thread then repeats the site's neighbour indices, the
// eight link loads and their widening to floats, work that a thread of the
// FP32 / FP16 hops, which are bound by instruction issue rather than HBM at
// 132 / 72 bytes per virtual site, pays for in issue slots.  Here N / C threads
// share a site; each computes the neighbour indices and loads and widens the
// eight links once, then runs the eight directions for its C right-hand sides
// r = t + k N / C (k = 0 .. C-1) one after the other, so that at each k the
// threads of a warp read contiguous runs of the neighbour blocks.  The
// arithmetic per right-hand side is that of the one-site kernels: the FP32
// hop's (agreement to rounding), the binary16 hop's with the projection in
// half2 (variants 14 / 15).
//
// Fused reductions (|out|^2 per right-hand side): a thread accumulates its C
// right-hand sides separately; at the end the block writes them to shared
// memory by (site slot, right-hand side) and re-reads them so that thread t
// holds a sum for right-hand side t mod N, the form the deterministic grid
// reduction takes.
#include "hr_hop_fam.h"
#include "hr_hop_x2.cuh"

using namespace hr;

namespace {

// one direction's term for right-hand side virtual site jn with the link q
// already widened
template <int MU, bool FWD, bool FIRST, bool NEG, int PREC>
__device__ __forceinline__ void chunk_term(const HopArgs &a, const float *nrm, int jn, const float (&q)[4],
                                           cpx<float> (&acc)[4][2])
{
    if constexpr (PREC == kF16) {
        const uint4 *sp = (const uint4 *)a.in;
        const uint4 w0 = __ldg(sp + vec_index(jn, 0, 2));
        const uint4 w1 = __ldg(sp + vec_index(jn, 1, 2));
        const float sc = __ldg(nrm + jn);
        h16_compute<MU, FWD, FIRST, NEG>(w0, w1, sc, q, acc);
    } else {
        cpx<float> s[4][2];
        float sc;
        load_spinor_raw<2, kF32>(a.in, a.g.nblk_s, jn, s, sc);
        hop_compute<MU, FWD, kRepFund, FIRST>(s, q, NEG, acc);
    }
}

template <int MU, bool NEG, int PREC>
__device__ __forceinline__ void chunk_dir(const HopArgs &a, const float *nrm, int l, int rr, const SiteNb &nb,
                                          const float (&q)[8][4], cpx<float> (&acc)[4][2])
{
    chunk_term<MU, true, MU == 0, NEG, PREC>(a, nrm, (nb.fwd[MU] << l) + rr, q[2 * MU], acc);
    chunk_term<MU, false, false, NEG, PREC>(a, nrm, (nb.bwd[MU] << l) + rr, q[2 * MU + 1], acc);
}

template <int PREC, int LC, int G5IN>
__device__ __forceinline__ void chunk_body(const HopArgs &a)
{
    constexpr int C = 1 << LC;
    constexpr bool NEG = G5IN != 0;
    if ((a.gate && *a.gate == 0.0) || (a.done && *a.done != 0.0)) return;
    const Geom &g = a.g;
    const int l = g.lrhs, lm = l - LC; // N / C = 2^lm threads per site
    const int nt = g.vh << lm;
    const int stride = gridDim.x * blockDim.x;
    const float *nrm =
        PREC == kF16 ? (const float *)((const char *)a.in + SpinorLayout<2, kF16>::data_bytes(g.nblk_s)) : nullptr;
    const float be = a.beta.h;
    const float bu = a.g5_out ? -be : be;
    const float al = a.alpha.h;
    float rs[C];
#pragma unroll
    for (int k = 0; k < C; ++k) rs[k] = 0.f;
    // the thread's right-hand sides: tp + k 2^lm (the stride is a multiple of 2^lm)
    const int tp = (blockIdx.x * blockDim.x + threadIdx.x) & ((1 << lm) - 1);
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < nt; u += stride) {
        const int i = u >> lm;
        SiteNb nb;
        site_neighbours(g, i, a.p, nb);
        float q[8][4];
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            load_quat<PREC>(a.gauge, g.nblk_g, a.p, mu, i, q[2 * mu]);
            load_quat<PREC>(a.gauge, g.nblk_g, 1 - a.p, mu, nb.bwd[mu], q[2 * mu + 1]);
        }
#pragma unroll 1
        for (int k = 0; k < C; ++k) {
            const int rr = tp + (k << lm);
            cpx<float> acc[4][2];
            chunk_dir<0, NEG, PREC>(a, nrm, l, rr, nb, q, acc);
            chunk_dir<1, NEG, PREC>(a, nrm, l, rr, nb, q, acc);
            chunk_dir<2, NEG, PREC>(a, nrm, l, rr, nb, q, acc);
            chunk_dir<3, NEG, PREC>(a, nrm, l, rr, nb, q, acc);
            SqAcc<float> red;
            hop_epilogue<PREC>(a, (i << l) + rr, acc, al, be, bu, red);
#pragma unroll
            for (int kk = 0; kk < C; ++kk)
                if (kk == k) rs[kk] += red.s;
        }
    }
    if (a.fin) {
        __shared__ double smem[32 * 32];
        __shared__ double sums[32];
        __shared__ double vals[256 * 4];
        const int t = threadIdx.x, n = g.nrhs;
        // site slot t >> lm of the block, right-hand side tp + k 2^lm
#pragma unroll
        for (int k = 0; k < C; ++k) vals[(t >> lm) * n + tp + (k << lm)] = (double)rs[k];
        __syncthreads();
        // thread t: right-hand side t mod N over the slots (t >> l) + s (B >> l), s < C
        double v = 0.0;
        const int per = blockDim.x >> l;
#pragma unroll
        for (int s = 0; s < C; ++s) v += vals[((t >> l) + s * per) * n + (t & (n - 1))];
        if (grid_reduce(v, n, a.red, sums, smem)) finish_reduction(a.fin, sums, n, a.scal);
    }
}

template <int PREC, int LC, int G5IN> __global__ void __launch_bounds__(256) k_hop_chunk(HopArgs a)
{
    chunk_body<PREC, LC, G5IN>(a);
}

template <int PREC>
void launch_chunk(const HopArgs &a, int lc, int grid, int block, cudaStream_t s)
{
    const bool g5 = a.g5_in != 0;
    if (lc == 1) (g5 ? k_hop_chunk<PREC, 1, 1> : k_hop_chunk<PREC, 1, 0>)<<<grid, block, 0, s>>>(a);
    else (g5 ? k_hop_chunk<PREC, 2, 1> : k_hop_chunk<PREC, 2, 0>)<<<grid, block, 0, s>>>(a);
}

} // namespace

namespace hr {

bool launch_hop_chunk(hr_ctx *ctx, const Geom &g, int rep, int prec, const HopArgs &a, HopChoice c, int,
                      cudaStream_t s, hr_status &st)
{
    const int lc = c.variant == kVarRhsChunk4 ? 2 : 1;
    if (rep != HR_FUND || (prec != kF32 && prec != kF16) || g.lrhs < lc) return false;
    // vals[] of the reduction holds blockDim x C doubles; whole warps
    if (c.block > 256 || c.block < 32 || (c.block & 31)) return false;
    const long long nt = (long long)g.vh << (g.lrhs - lc);
    const int grid = grid_for(nt, c.block, a.fin ? kMaxBlocks : (1 << 30));
    if (prec == kF32) launch_chunk<kF32>(a, lc, grid, c.block, s);
    else launch_chunk<kF16>(a, lc, grid, c.block, s);
    st = check_launch(ctx, "right-hand-side chunk hop kernel");
    return true;
}

} // namespace hr
