// hr_hop_dev.cuh -- device code of the Wilson hop shared by the single-lattice
// kernels (hr_hop.cu) and the batched persistent solver (hr_batch.cu): the launch
// arguments, one direction's projection / colour multiplication / accumulation,
// and the epilogue out = alpha aux + beta [g5] H [g5] in with the fused |out|^2.
#pragma once

#include "hr_clover.cuh"
#include "hr_host.h"

namespace hr {

struct HopArgs {
    Geom g;
    int p;
    const void *gauge;
    const void *in;
    const void *aux;
    void *out;
    coef2 alpha, beta;
    int beta_pow2; // beta is a power of two and there is no aux: exact scaling
    int g5_in, g5_out;
    int fin;
    RedSlot red;
    double *scal;
    const double *gate;
    const double *done; // skip all work when *done != 0 (solver converged)
    float unit, nil;    // 1 and 0, passed at run time so the compiler keeps the
                        // +-1 multipliers of the packed-FMA additions as FMAs
    void *cg_x;         // fused CG update (cg_r != nullptr): x += alpha p,
    const void *cg_p;   // r -= alpha out, |r|^2 reduced; out is not stored
    void *cg_r;
    long long wait_cycles; // bound of a device wait (tiled kernels' bulk copies)
    int inject_no_copy;    // failure injection for tests: announce the tiled
                           // kernels' copies but never queue them
    const void *clov;      // clover half-field of the output parity (kClovAux / kClovOut), or nullptr
    int clov_mode;
};



__device__ __forceinline__ dd mul_pow2(dd x, float s) { return dd(x.h * s, x.l * s); }
__device__ __forceinline__ float mul_pow2(float x, float s) { return x * s; }

// projection, colour multiplication and accumulation of one direction
template <int MU, bool FWD, int REP, bool FIRST = false, class T, int NC, class LINK>
__device__ __forceinline__ void hop_compute(cpx<T> (&s)[4][NC], const LINK &link, bool neg_upper,
                                            cpx<T> (&acc)[4][NC])
{
    if (neg_upper) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            s[0][c] = {-s[0][c].re, -s[0][c].im};
            s[1][c] = {-s[1][c].re, -s[1][c].im};
        }
    }
    cpx<T> h[2][NC], r[2][NC];
    spin_project<MU, FWD>(s, h);
    if constexpr (REP == kRepFund) {
        su2_mul<!FWD>(link, h[0], r[0]);
        su2_mul<!FWD>(link, h[1], r[1]);
    } else {
        so3_mul<!FWD>(link, h[0], r[0]);
        so3_mul<!FWD>(link, h[1], r[1]);
    }
    spin_accumulate<MU, FWD, T, NC, FIRST>(acc, r);
}

// one direction's term for a neighbour spinor s already loaded (binary16: s
// unscaled, sc its scale; the projection and the colour product are linear, so
// the scale multiplies the link instead, 4 or 9 numbers)
template <int MU, bool FWD, int REP, int PREC, bool FIRST = false, class T, int NC>
__device__ __forceinline__ void hop_term_with(const HopArgs &a, int site_link, int link_par, cpx<T> (&s)[4][NC],
                                              float sc, bool neg_upper, cpx<T> (&acc)[4][NC])
{
    if constexpr (REP == kRepFund) {
        T q[4];
        load_quat<PREC>(a.gauge, a.g.nblk_g, link_par, MU, site_link, q);
        if constexpr (PREC == kF16) {
#pragma unroll
            for (int k = 0; k < 4; ++k) q[k] = q[k] * sc;
        }
        hop_compute<MU, FWD, REP, FIRST>(s, q, neg_upper, acc);
    } else {
        T R[3][3];
        if constexpr (REP == kRepAdj) {
            T q[4];
            load_quat<PREC>(a.gauge, a.g.nblk_g, link_par, MU, site_link, q);
            quat_to_adj(q, R);
        } else {
            load_mat<PREC>(a.gauge, a.g.nblk_g, link_par, MU, site_link, R);
        }
        if constexpr (PREC == kF16) {
#pragma unroll
            for (int k = 0; k < 9; ++k) R[k / 3][k % 3] = R[k / 3][k % 3] * sc;
        }
        hop_compute<MU, FWD, REP, FIRST>(s, R, neg_upper, acc);
    }
}

template <int MU, bool FWD, int REP, int PREC, bool FIRST = false, class T, int NC>
__device__ __forceinline__ void hop_term(const HopArgs &a, int site_link, int link_par, int j_nb, bool neg_upper,
                                         cpx<T> (&acc)[4][NC])
{
    cpx<T> s[4][NC];
    float sc;
    load_spinor_raw<NC, PREC>(a.in, a.g.nblk_s, j_nb, s, sc);
    hop_term_with<MU, FWD, REP, PREC, FIRST>(a, site_link, link_par, s, sc, neg_upper, acc);
}

// G5IN: 0 / 1 = the input is (not) multiplied by g5, fixed at compile time;
// -1 = read a.g5_in at run time
template <int G5IN> __device__ __forceinline__ bool g5_in_of(const HopArgs &a)
{
    if constexpr (G5IN < 0) return a.g5_in != 0;
    else return G5IN != 0;
}

template <int MU, int REP, int PREC, int G5IN, bool FIRST = false, class T, int NC>
__device__ __forceinline__ void hop_dir(const HopArgs &a, int i, int rr, const SiteNb &nb, cpx<T> (&acc)[4][NC])
{
    const int l = a.g.lrhs;
    // forward: (1 - g_mu) U_mu(x) psi(x + mu); the link sits at x (parity p)
    hop_term<MU, true, REP, PREC, FIRST>(a, i, a.p, (nb.fwd[MU] << l) + rr, g5_in_of<G5IN>(a), acc);
    // backward: (1 + g_mu) U_mu(x - mu)^+ psi(x - mu); the link sits at x - mu (parity 1-p)
    hop_term<MU, false, REP, PREC>(a, nb.bwd[MU], 1 - a.p, (nb.bwd[MU] << l) + rr, g5_in_of<G5IN>(a), acc);
}

// The epilogue's own operands -- the aux vector, and the fused CG update's
// x, p and r -- are read only after the eight directions, so their load
// latency would add to every site of the reducing hops.  Requested into L1
// when the site starts, they arrive behind the directions' work (a hint: no
// effect on the results).
__device__ __forceinline__ void prefetch_l1(const void *p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }
template <int NC, int PREC>
__device__ __forceinline__ void prefetch_site(const void *base, int nblk_s, int j)
{
    constexpr int NV = SpinorLayout<NC, PREC>::NVEC;
    const uint4 *v = (const uint4 *)base;
#pragma unroll
    for (int k = 0; k < NV; ++k) prefetch_l1(v + vec_index(j, k, NV));
    if constexpr (PREC == kF16) prefetch_l1((const float *)((const char *)base + SpinorLayout<NC, PREC>::data_bytes(nblk_s)) + j);
}
template <int NC, int PREC>
__device__ __forceinline__ void epilogue_prefetch(const HopArgs &a, int j)
{
    // the solvers' hot path is the fundamental one; with three colours the
    // four fields are 24 vectors a site, and the adjoint plain hop ran slower
    // with the request code in it
    if constexpr (NC != 2) return;
    if (a.aux) prefetch_site<NC, PREC>(a.aux, a.g.nblk_s, j);
    if (a.cg_r) {
        prefetch_site<NC, PREC == kF16 ? kF32 : PREC>(a.cg_x, a.g.nblk_s, j);
        prefetch_site<NC, PREC>(a.cg_p, a.g.nblk_s, j);
        prefetch_site<NC, PREC>(a.cg_r, a.g.nblk_s, j);
    }
}

// out = alpha * aux + beta * g5^{g5_out} acc, stored; |out|^2 into red.
// CLOV: the kernel instantiation that also applies the clover site term
// (a.clov_mode); the others carry no trace of it.
template <int PREC, bool CLOV = false, class T, int NC>
__device__ __forceinline__ void hop_epilogue(const HopArgs &a, int j, const cpx<T> (&acc)[4][NC], T al, T be, T bu,
                                             SqAcc<T> &red)
{
    constexpr int CP = clover_prec(PREC);
    cpx<T> o[4][NC];
    if (a.aux) {
        load_spinor<NC, PREC>(a.aux, a.g.nblk_s, j, o);
        if constexpr (CLOV)
            if (a.clov_mode == kClovAux) clover_apply<CP>(a.clov, j >> a.g.lrhs, o);
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                T b = s < 2 ? bu : be;
                o[s][c] = {al * o[s][c].re + b * acc[s][c].re, al * o[s][c].im + b * acc[s][c].im};
            }
    } else if (a.beta_pow2) {
        const float bh = a.g5_out ? -a.beta.h : a.beta.h;
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                float b = s < 2 ? bh : a.beta.h;
                o[s][c] = {mul_pow2(acc[s][c].re, b), mul_pow2(acc[s][c].im, b)};
            }
    } else {
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                T b = s < 2 ? bu : be;
                o[s][c] = {b * acc[s][c].re, b * acc[s][c].im};
            }
    }
    if constexpr (CLOV)
        if (a.clov_mode == kClovOut) clover_apply<CP>(a.clov, j >> a.g.lrhs, o);
    if (a.cg_r) {
        // the CG's x/r update on this site, with q = o in registers (the
        // vector kernel's arithmetic, in the hop's precision); the binary16
        // solver keeps its x increment in FP32, and r -= alpha q takes q
        // before any rounding to binary16
        constexpr int PX = PREC == kF16 ? kF32 : PREC;
        const T alr = Real<T>::from_double(a.scal[S_ALPHA * kMaxRhsSlots + (j & (a.g.nrhs - 1))]);
        cpx<T> xv[4][NC], pv[4][NC], rv[4][NC];
        load_spinor<NC, PX>(a.cg_x, a.g.nblk_s, j, xv);
        load_spinor<NC, PREC>(a.cg_p, a.g.nblk_s, j, pv);
        load_spinor<NC, PREC>(a.cg_r, a.g.nblk_s, j, rv);
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                xv[s][c].re += alr * pv[s][c].re;
                xv[s][c].im += alr * pv[s][c].im;
                rv[s][c].re -= alr * o[s][c].re;
                rv[s][c].im -= alr * o[s][c].im;
                red.add(rv[s][c].re);
                red.add(rv[s][c].im);
            }
        store_spinor<NC, PX>(a.cg_x, a.g.nblk_s, j, xv);
        store_spinor<NC, PREC>(a.cg_r, a.g.nblk_s, j, rv);
        return;
    }
    store_spinor<NC, PREC>(a.out, a.g.nblk_s, j, o);
    if (a.fin) {
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                red.add(o[s][c].re);
                red.add(o[s][c].im);
            }
    }
}

// one output site j (virtual index) of the unrolled hop: all 8 directions and the epilogue
template <int REP, int PREC, int G5IN = -1, bool CLOV = false, class T>
__device__ __forceinline__ void hop_site(const HopArgs &a, int j, T al, T be, T bu, SqAcc<T> &red)
{
    constexpr int NC = RepTraits<REP>::NC;
    const Geom &g = a.g;
    const int i = j >> g.lrhs, rr = j & (g.nrhs - 1);
    SiteNb nb;
    site_neighbours(g, i, a.p, nb);
    epilogue_prefetch<NC, PREC>(a, j);
    cpx<T> acc[4][NC]; // set by the first term
    hop_dir<0, REP, PREC, G5IN, true>(a, i, rr, nb, acc);
    hop_dir<1, REP, PREC, G5IN>(a, i, rr, nb, acc);
    hop_dir<2, REP, PREC, G5IN>(a, i, rr, nb, acc);
    hop_dir<3, REP, PREC, G5IN>(a, i, rr, nb, acc);
    hop_epilogue<PREC, CLOV>(a, j, acc, al, be, bu, red);
}

} // namespace hr
