// hr_hop_twist.cu -- the hop for lattices with twisted fermion boundary
// conditions, psi(x + L_mu mu) = e^{i theta_mu} psi(x): a hop that reaches its
// neighbour forward across the boundary of direction mu multiplies the
// spinor by e^{+i theta_mu}, backward by e^{-i theta_mu} (the phase commutes
// with the spin projection and the colour product, so it is applied to the
// projected half spinor, 2 NC complex products).  An SU(2) link times a phase is no
// quaternion, so the twist cannot ride in the packed links as the
// antiperiodic sign does (that sign stays there and combines with the phase).
//
// One thread per output (virtual) site, the operand loads, projection, colour
// product and epilogue of the plain kernel (hr_hop_dev.cuh), every operator
// mode of HopArgs (Schur epilogues, fused CG update, |out|^2 reduction, clover
// site term); for the fundamental FP64 hop the paired double-float arithmetic
// of the tuned kernels (two colours per f32x2 instruction) instead.  Twisted
// lattices always run these kernels: the dispatch sends them here before
// consulting the autotuned variant, so the tuned kernels of untwisted
// lattices carry no trace of the twist.
#include "hr_host.h"
#include "hr_hop_dev.cuh"
#include "hr_hop_fam.h"
#include "hr_hop_x2.cuh"

using namespace hr;

namespace {

// coordinates x_mu of the site with even-odd index i and parity p
__device__ __forceinline__ void site_coords(const Geom &g, int i, int p, int (&x)[4])
{
    const int row = fdiv(i, g.div_h3);
    const int k = i - row * g.h3;
    const int r1 = fdiv(row, g.div_d2);
    x[2] = row - r1 * g.d[2];
    x[0] = fdiv(r1, g.div_d1);
    x[1] = r1 - x[0] * g.d[1];
    x[3] = 2 * k + ((x[0] + x[1] + x[2] + p) & 1);
}

// h *= c + i sn (the projected half spinor)
template <class T, int NC> __device__ __forceinline__ void phase_half(cpx<T> (&h)[2][NC], T c, T sn)
{
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < NC; ++b) h[a][b] = {h[a][b].re * c - h[a][b].im * sn, h[a][b].re * sn + h[a][b].im * c};
}

// one hop term of the twisted kernel: as hop_term_with / hop_compute, with the
// boundary phase (e^{+-i theta}) on the projected half spinor when `cross`
template <int MU, bool FWD, int REP, int PREC, bool FIRST, class T, int NC>
__device__ __forceinline__ void twisted_term(const HopArgs &a, int site_link, int link_par, cpx<T> (&s)[4][NC],
                                             float sc, bool neg_upper, bool cross, T c, T sn,
                                             cpx<T> (&acc)[4][NC])
{
    if (neg_upper) {
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            s[0][k] = {-s[0][k].re, -s[0][k].im};
            s[1][k] = {-s[1][k].re, -s[1][k].im};
        }
    }
    cpx<T> h[2][NC], r[2][NC];
    spin_project<MU, FWD>(s, h);
    if (cross) phase_half(h, c, sn);
    if constexpr (REP == kRepFund) {
        T q[4];
        load_quat<PREC>(a.gauge, a.g.nblk_g, link_par, MU, site_link, q);
        if constexpr (PREC == kF16) {
#pragma unroll
            for (int k = 0; k < 4; ++k) q[k] = q[k] * sc;
        }
        su2_mul<!FWD>(q, h[0], r[0]);
        su2_mul<!FWD>(q, h[1], r[1]);
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
        so3_mul<!FWD>(R, h[0], r[0]);
        so3_mul<!FWD>(R, h[1], r[1]);
    }
    spin_accumulate<MU, FWD, T, NC, FIRST>(acc, r);
}

template <int MU, int REP, int PREC, bool FIRST, class T, int NC>
__device__ __forceinline__ void twisted_dir(const HopArgs &a, int i, int rr, const SiteNb &nb, const int (&x)[4],
                                            cpx<T> (&acc)[4][NC])
{
    const Geom &g = a.g;
    const int l = g.lrhs;
    const bool g5 = a.g5_in != 0;
    // directions without a twist skip the phase (a uniform test: no divergence)
    const bool tw = g.tw_s[MU].h != 0.f || g.tw_s[MU].l != 0.f || g.tw_c[MU].h != 1.f || g.tw_c[MU].l != 0.f;
    const T c = Real<T>::from_coef(g.tw_c[MU]), sn = Real<T>::from_coef(g.tw_s[MU]);
    cpx<T> s[4][NC];
    float sc;
    // forward: (1 - g_mu) U_mu(x) psi(x + mu), e^{+i theta} across the boundary
    load_spinor_raw<NC, PREC>(a.in, g.nblk_s, (nb.fwd[MU] << l) + rr, s, sc);
    twisted_term<MU, true, REP, PREC, FIRST>(a, i, a.p, s, sc, g5, tw && x[MU] == g.d[MU] - 1, c, sn, acc);
    // backward: (1 + g_mu) U_mu(x - mu)^+ psi(x - mu), e^{-i theta} across it
    load_spinor_raw<NC, PREC>(a.in, g.nblk_s, (nb.bwd[MU] << l) + rr, s, sc);
    twisted_term<MU, false, REP, PREC, false>(a, nb.bwd[MU], 1 - a.p, s, sc, g5, tw && x[MU] == 0, c, -sn, acc);
}

template <int REP, int PREC, bool CLOV>
__global__ void __launch_bounds__(128) k_hop_twist(HopArgs a)
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
        int x[4];
        site_coords(g, i, a.p, x);
        cpx<T> acc[4][NC];
        twisted_dir<0, REP, PREC, true>(a, i, rr, nb, x, acc);
        twisted_dir<1, REP, PREC, false>(a, i, rr, nb, x, acc);
        twisted_dir<2, REP, PREC, false>(a, i, rr, nb, x, acc);
        twisted_dir<3, REP, PREC, false>(a, i, rr, nb, x, acc);
        hop_epilogue<PREC, CLOV>(a, j, acc, al, be, bu, red);
    }
    if (a.fin) {
        __shared__ double smem[32 * 32];
        __shared__ double sums[32];
        if (grid_reduce(red, g.nrhs, a.red, sums, smem)) finish_reduction(a.fin, sums, g.nrhs, a.scal);
    }
}

// ---- fundamental FP64: the paired double-float arithmetic of the tuned
// kernels (two colours per f32x2 instruction, hr_hop_x2.cuh) with the phase on
// the projected doublets.  The kernel carries the same operator modes.

// h *= (c + i s) on colour doublets: re' = c re - s im, im' = s re + c im
// (C, S: c and s in both lanes; cn, sn: their negated hi parts)
__device__ __forceinline__ cdd2 phase_x2(const K2 &k, const cdd2 &h, const dd2 &C, float2 cn, const dd2 &S,
                                         float2 sn)
{
    cdd2 r;
    r.re = first_prod2<1>(k, mul2(k, C, cn, h.re));
    r.re = acc_prod2<-1>(k, r.re, mul2(k, S, sn, h.im));
    r.im = first_prod2<1>(k, mul2(k, S, sn, h.re));
    r.im = acc_prod2<1>(k, r.im, mul2(k, C, cn, h.im));
    return r;
}

template <int MU, bool FWD, bool FIRST, bool NEG>
__device__ __forceinline__ void x2t_term(const HopArgs &a, const K2 &k, int site_link, int link_par, int j_nb,
                                         bool cross, const dd2 &C, float2 cn, const dd2 &S, float2 sn,
                                         cdd2 (&acc)[4])
{
    using D = X2Dir<MU, FWD>;
    constexpr int F = NEG ? 2 : 0;
    const float4 *sp = (const float4 *)a.in;
    float4 w[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) w[v] = __ldg(sp + vec_index(j_nb, v, 8));
    const size_t slot = (size_t)(link_par * 4 + MU) * a.g.nblk_g + (site_link >> 5);
    const float4 *qp = (const float4 *)a.gauge;
    const float4 qh = __ldg(qp + (slot * 2 + 0) * 32 + (site_link & 31));
    const float4 ql = __ldg(qp + (slot * 2 + 1) * 32 + (site_link & 31));
    cdd2 sv[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        sv[t].re = {make_float2(w[2 * t].x, w[2 * t].y), make_float2(w[2 * t + 1].x, w[2 * t + 1].y)};
        sv[t].im = {make_float2(w[2 * t].z, w[2 * t].w), make_float2(w[2 * t + 1].z, w[2 * t + 1].w)};
    }
    cdd2 h0 = cadd_pow_i<(D::c0 + F) & 3>(k, sv[0], sv[D::pi0]);
    cdd2 h1 = cadd_pow_i<(D::c1 + F) & 3>(k, sv[1], sv[D::pi1]);
    if (cross) {
        h0 = phase_x2(k, h0, C, cn, S, sn);
        h1 = phase_x2(k, h1, C, cn, S, sn);
    }
    const Link2 U = link2(qh, ql);
    x2_rebuild<0, D, F, FIRST>(k, su2_x2<FWD>(k, U, h0), acc);
    x2_rebuild<1, D, F, FIRST>(k, su2_x2<FWD>(k, U, h1), acc);
}

template <int MU, bool FIRST, bool NEG>
__device__ __forceinline__ void x2t_dir(const HopArgs &a, const K2 &k, int i, int rr, const SiteNb &nb,
                                        const int (&x)[4], cdd2 (&acc)[4])
{
    const Geom &g = a.g;
    const int l = g.lrhs;
    const bool tw = g.tw_s[MU].h != 0.f || g.tw_s[MU].l != 0.f || g.tw_c[MU].h != 1.f || g.tw_c[MU].l != 0.f;
    const dd c = Real<dd>::from_coef(g.tw_c[MU]), sn = Real<dd>::from_coef(g.tw_s[MU]);
    const dd2 C = {make_float2(c.h, c.h), make_float2(c.l, c.l)};
    const float2 cn = make_float2(-c.h, -c.h);
    // forward across the boundary e^{+i theta}, backward e^{-i theta}
    const dd2 Sf = {make_float2(sn.h, sn.h), make_float2(sn.l, sn.l)};
    const dd2 Sb = {make_float2(-sn.h, -sn.h), make_float2(-sn.l, -sn.l)};
    x2t_term<MU, true, FIRST, NEG>(a, k, i, a.p, (nb.fwd[MU] << l) + rr, tw && x[MU] == g.d[MU] - 1, C, cn, Sf,
                                   make_float2(-sn.h, -sn.h), acc);
    x2t_term<MU, false, false, NEG>(a, k, nb.bwd[MU], 1 - a.p, (nb.bwd[MU] << l) + rr, tw && x[MU] == 0, C, cn, Sb,
                                    make_float2(sn.h, sn.h), acc);
}

template <int G5IN, bool CLOV>
__device__ __forceinline__ void x2t_body(const HopArgs &a)
{
    constexpr bool NEG = G5IN != 0;
    if ((a.gate && *a.gate == 0.0) || (a.done && *a.done != 0.0)) return;
    const K2 k = make_k2(a.unit, a.nil);
    const Geom &g = a.g;
    const int nv = g.vh << g.lrhs;
    const int stride = gridDim.x * blockDim.x;
    const dd be = Real<dd>::from_coef(a.beta);
    const dd bu = a.g5_out ? -be : be;
    const dd al = Real<dd>::from_coef(a.alpha);
    SqAcc<dd> red;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nv; j += stride) {
        const int i = j >> g.lrhs, rr = j & (g.nrhs - 1);
        SiteNb nb;
        site_neighbours(g, i, a.p, nb);
        int x[4];
        site_coords(g, i, a.p, x);
        cdd2 acc[4];
        x2t_dir<0, true, NEG>(a, k, i, rr, nb, x, acc);
        x2t_dir<1, false, NEG>(a, k, i, rr, nb, x, acc);
        x2t_dir<2, false, NEG>(a, k, i, rr, nb, x, acc);
        x2t_dir<3, false, NEG>(a, k, i, rr, nb, x, acc);
        x2_epilogue<CLOV>(a, j, acc, al, be, bu, red);
    }
    if (a.fin) {
        __shared__ double smem[32 * 32];
        __shared__ double sums[32];
        if (grid_reduce(red, g.nrhs, a.red, sums, smem)) finish_reduction(a.fin, sums, g.nrhs, a.scal);
    }
}

template <int G5IN, bool CLOV> __global__ void __maxnreg__(128) k_hop_x2t(HopArgs a) { x2t_body<G5IN, CLOV>(a); }

template <int REP, int PREC> struct TwistLaunch {
    static bool run(hr_ctx *ctx, const HopArgs &a, int grid, cudaStream_t s, hr_status &st)
    {
        if constexpr (REP == kRepFund && PREC == kF64) {
            const bool g5 = a.g5_in != 0, clov = a.clov_mode != kClovNone;
            if (clov) (g5 ? k_hop_x2t<1, true> : k_hop_x2t<0, true>)<<<grid, kTwistBlock, 0, s>>>(a);
            else (g5 ? k_hop_x2t<1, false> : k_hop_x2t<0, false>)<<<grid, kTwistBlock, 0, s>>>(a);
            st = check_launch(ctx, "paired hop kernel (twisted boundaries)");
            return true;
        }
        if (a.clov_mode != kClovNone) k_hop_twist<REP, PREC, true><<<grid, kTwistBlock, 0, s>>>(a);
        else k_hop_twist<REP, PREC, false><<<grid, kTwistBlock, 0, s>>>(a);
        st = check_launch(ctx, "hop kernel (twisted boundaries)");
        return true;
    }
};

} // namespace

namespace hr {

void launch_hop_twisted(hr_ctx *ctx, int rep, int prec, const HopArgs &a, cudaStream_t s, hr_status &st)
{
    const long long nv = (long long)a.g.vh << a.g.lrhs;
    const int grid = grid_for(nv, kTwistBlock, a.fin ? kMaxBlocks : (1 << 30));
    if (!for_config<TwistLaunch>(rep, prec, ctx, a, grid, s, st))
        st = set_error(ctx, HR_ERR_INVALID_ARG, "bad rep/prec");
}

} // namespace hr
