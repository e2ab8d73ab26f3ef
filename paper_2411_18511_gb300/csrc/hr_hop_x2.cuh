// hr_hop_x2.cuh -- double-float arithmetic on packed f32x2 FMAs for the
// fundamental hop, shared by the paired hop kernels (hr_hop_x2.cu) and the
// batched solver (hr_batch.cu).
#pragma once

#include "hr_hop_dev.cuh"

namespace hr {

// ---------------------------------------------------------------- paired (f32x2) variant
// The fundamental double-float hop on the packed FP32x2 FMA of sm_100 and later
// (__ffma2_rn: two lanes per instruction, the same lane rate as scalar FFMA).
// The lanes are the two colours: the FP64 layout keeps, per spin, the hi parts
// (c0.re, c1.re, c0.im, c1.im) in one vector and the lo parts in the next, so
// each loaded vector is two ready lane pairs.  The projection and the rebuild
// of the lower spins treat both colours alike (a factor i only swaps which
// pair is re and which im); the SU(2) product mixes the colours through one
// lane swap of h.  Every addition is an FMA with a +-1 multiplier -- the packed
// add has a lower rate -- so the FP32 pipes do the scalar kernel's operations
// in half the instructions: the double-float hop is no longer issue-bound.
// Each sum is formed in the scalar kernel's order, and rounding is symmetric
// under negation, so the results are bit-identical to the scalar kernels.

struct dd2 {
    float2 h, l; // two double-float numbers: lanes x and y
};
struct cdd2 {
    dd2 re, im; // a colour doublet of complex numbers
};
struct K2 {
    float2 one, mone, zero; // (1, 1), (-1, -1), (0, 0)
    float2 mp, pm;          // (-1, 1), (1, -1): a factor i or -i on (re, im) lanes
};
// the constants from run-time 1 and 0, so that the compiler keeps them as FMA operands
__device__ __forceinline__ K2 make_k2(float unit, float nil)
{
    return {make_float2(unit, unit), make_float2(-unit, -unit), make_float2(nil, nil), make_float2(-unit, unit),
            make_float2(unit, -unit)};
}

// a + sg b lane by lane, sg a pair of +-1 (Knuth's TwoSum on the hi parts, lo parts added)
__device__ __forceinline__ dd2 add2v(const K2 &k, const dd2 &a, const dd2 &b, float2 sg)
{
    const float2 s = __ffma2_rn(b.h, sg, a.h);   // fl(a + sg b)
    const float2 w = __ffma2_rn(s, k.mone, a.h); // a - s, exact
    const float2 t = __ffma2_rn(w, k.one, s);    // the part of s that came from a
    const float2 da = __ffma2_rn(t, k.mone, a.h);
    const float2 db = __ffma2_rn(b.h, sg, w);
    const float2 e = __ffma2_rn(da, k.one, db);
    const float2 lo = __ffma2_rn(b.l, sg, a.l);
    return {s, __ffma2_rn(e, k.one, lo)};
}

// a + S b on both lanes
template <int S> __device__ __forceinline__ dd2 add2(const K2 &k, const dd2 &a, const dd2 &b)
{
    return add2v(k, a, b, S > 0 ? k.one : k.mone);
}

// c x = -P + L: P = fl(-c.h x.h) exactly, L = the product's rounding error
// (TwoProduct by FMA) plus the cross terms c.h x.l + c.l x.h; cnh = -c.h
struct prod2 {
    float2 P, L;
};
__device__ __forceinline__ prod2 mul2(const K2 &k, const dd2 &c, float2 cnh, const dd2 &x)
{
    const float2 P = __ffma2_rn(cnh, x.h, k.zero);
    float2 e = __ffma2_rn(c.h, x.h, P);
    e = __ffma2_rn(c.h, x.l, e);
    e = __ffma2_rn(c.l, x.h, e);
    return {P, e};
}
// r + S c x
template <int S> __device__ __forceinline__ dd2 acc_prod2(const K2 &k, const dd2 &r, const prod2 &p)
{
    dd2 b{p.P, p.L}; // r + S (-P) on the hi parts, r + S L on the lo parts
    const float2 sgh = S > 0 ? k.mone : k.one, sgl = S > 0 ? k.one : k.mone;
    const float2 s = __ffma2_rn(b.h, sgh, r.h);
    const float2 w = __ffma2_rn(s, k.mone, r.h);
    const float2 t = __ffma2_rn(w, k.one, s);
    const float2 da = __ffma2_rn(t, k.mone, r.h);
    const float2 db = __ffma2_rn(b.h, sgh, w);
    const float2 e = __ffma2_rn(da, k.one, db);
    const float2 lo = __ffma2_rn(b.l, sgl, r.l);
    return {s, __ffma2_rn(e, k.one, lo)};
}
// S c x as a double-float pair
template <int S> __device__ __forceinline__ dd2 first_prod2(const K2 &k, const prod2 &p)
{
    if constexpr (S > 0) return {__ffma2_rn(p.P, k.mone, k.zero), p.L};
    else return {p.P, __ffma2_rn(p.L, k.mone, k.zero)};
}

__device__ __forceinline__ dd2 neg2(const K2 &k, const dd2 &a)
{
    return {__ffma2_rn(a.h, k.mone, k.zero), __ffma2_rn(a.l, k.mone, k.zero)};
}
__device__ __forceinline__ float2 swap2(float2 v) { return make_float2(v.y, v.x); }
__device__ __forceinline__ dd2 swap2(const dd2 &v) { return {swap2(v.h), swap2(v.l)}; }

// x + i^C y (C = 0: +1, 1: +i, 2: -1, 3: -i) for colour doublets
template <int C> __device__ __forceinline__ cdd2 cadd_pow_i(const K2 &k, const cdd2 &x, const cdd2 &y)
{
    if constexpr (C == 0) return {add2<1>(k, x.re, y.re), add2<1>(k, x.im, y.im)};
    else if constexpr (C == 1) return {add2<-1>(k, x.re, y.im), add2<1>(k, x.im, y.re)};
    else if constexpr (C == 2) return {add2<-1>(k, x.re, y.re), add2<-1>(k, x.im, y.im)};
    else return {add2<1>(k, x.re, y.im), add2<-1>(k, x.im, y.re)};
}
// i^C y
template <int C> __device__ __forceinline__ cdd2 pow_i(const K2 &k, const cdd2 &y)
{
    if constexpr (C == 0) return y;
    else if constexpr (C == 1) return {neg2(k, y.im), y.re};
    else if constexpr (C == 2) return {neg2(k, y.re), neg2(k, y.im)};
    else return {y.im, neg2(k, y.re)};
}

// chiral-basis (1 -/+ g_mu): h_t = s_t + i^{c_t} s_{pi_t} (t = 0, 1) and the
// rebuilt lower spins acc_{2+u} += i^{d_u} r_{rho_u} (u = 0, 1)
template <int MU, bool FWD> struct X2Dir;
template <> struct X2Dir<0, true> { static constexpr int c0 = 2, pi0 = 2, c1 = 2, pi1 = 3, d0 = 2, rho0 = 0, d1 = 2, rho1 = 1; };
template <> struct X2Dir<0, false> { static constexpr int c0 = 0, pi0 = 2, c1 = 0, pi1 = 3, d0 = 0, rho0 = 0, d1 = 0, rho1 = 1; };
template <> struct X2Dir<1, true> { static constexpr int c0 = 1, pi0 = 3, c1 = 1, pi1 = 2, d0 = 3, rho0 = 1, d1 = 3, rho1 = 0; };
template <> struct X2Dir<1, false> { static constexpr int c0 = 3, pi0 = 3, c1 = 3, pi1 = 2, d0 = 1, rho0 = 1, d1 = 1, rho1 = 0; };
template <> struct X2Dir<2, true> { static constexpr int c0 = 0, pi0 = 3, c1 = 2, pi1 = 2, d0 = 2, rho0 = 1, d1 = 0, rho1 = 0; };
template <> struct X2Dir<2, false> { static constexpr int c0 = 2, pi0 = 3, c1 = 0, pi1 = 2, d0 = 0, rho0 = 1, d1 = 2, rho1 = 0; };
template <> struct X2Dir<3, true> { static constexpr int c0 = 1, pi0 = 2, c1 = 3, pi1 = 3, d0 = 3, rho0 = 0, d1 = 1, rho1 = 1; };
template <> struct X2Dir<3, false> { static constexpr int c0 = 3, pi0 = 2, c1 = 1, pi1 = 3, d0 = 1, rho0 = 0, d1 = 3, rho1 = 1; };

// link coefficient pairs over the colour lanes: U h = (C0 + i C3) h + (C2 + i C1) swap(h)
// with C0 = (a0, a0), C1 = (a1, a1), C2 = (a2, -a2), C3 = (a3, -a3); cn* = -C*.h
struct Link2 {
    dd2 c0, c1, c2, c3;
    float2 n0, n1, n2, n3;
};
__device__ __forceinline__ Link2 link2(const float4 &qh, const float4 &ql)
{
    Link2 L;
    L.c0 = {make_float2(qh.x, qh.x), make_float2(ql.x, ql.x)};
    L.c1 = {make_float2(qh.y, qh.y), make_float2(ql.y, ql.y)};
    L.c2 = {make_float2(qh.z, -qh.z), make_float2(ql.z, -ql.z)};
    L.c3 = {make_float2(qh.w, -qh.w), make_float2(ql.w, -ql.w)};
    L.n0 = make_float2(-qh.x, -qh.x);
    L.n1 = make_float2(-qh.y, -qh.y);
    L.n2 = make_float2(-qh.z, qh.z);
    L.n3 = make_float2(-qh.w, qh.w);
    return L;
}

// r = U h (FWD) or U^+ h, in the scalar kernel's order of terms:
//   U:   re = C0 hr - C3 hi + C2 sr - C1 si,  im = C0 hi + C3 hr + C2 si + C1 sr
//   U^+: re = C0 hr + C3 hi - C2 sr + C1 si,  im = C0 hi - C3 hr - C2 si - C1 sr
// (s = swap(h))
template <bool FWD> __device__ __forceinline__ cdd2 su2_x2(const K2 &k, const Link2 &U, const cdd2 &h)
{
    constexpr int S = FWD ? 1 : -1;
    const dd2 sr = swap2(h.re), si = swap2(h.im);
    cdd2 r;
    r.re = first_prod2<1>(k, mul2(k, U.c0, U.n0, h.re));
    r.re = acc_prod2<-S>(k, r.re, mul2(k, U.c3, U.n3, h.im));
    r.re = acc_prod2<S>(k, r.re, mul2(k, U.c2, U.n2, sr));
    r.re = acc_prod2<-S>(k, r.re, mul2(k, U.c1, U.n1, si));
    r.im = first_prod2<1>(k, mul2(k, U.c0, U.n0, h.im));
    r.im = acc_prod2<S>(k, r.im, mul2(k, U.c3, U.n3, h.re));
    r.im = acc_prod2<S>(k, r.im, mul2(k, U.c2, U.n2, si));
    r.im = acc_prod2<S>(k, r.im, mul2(k, U.c1, U.n1, sr));
    return r;
}

// one direction: acc (+)= (1 -/+ g_mu) U psi(neighbour) in doublet form.  NEG:
// the input's upper spins are negated (g5 in), folded into the signs.
// acc_t (+)= i^F r_t and acc_{2+u} (+)= i^{d_u + F} r_t for the u with rho_u = t
template <int T, class D, int F, bool FIRST>
__device__ __forceinline__ void x2_rebuild(const K2 &k, const cdd2 &r, cdd2 (&acc)[4])
{
    if constexpr (FIRST) acc[T] = pow_i<F>(k, r);
    else acc[T] = cadd_pow_i<F>(k, acc[T], r);
    if constexpr (D::rho0 == T) {
        if constexpr (FIRST) acc[2] = pow_i<(D::d0 + F) & 3>(k, r);
        else acc[2] = cadd_pow_i<(D::d0 + F) & 3>(k, acc[2], r);
    }
    if constexpr (D::rho1 == T) {
        if constexpr (FIRST) acc[3] = pow_i<(D::d1 + F) & 3>(k, r);
        else acc[3] = cadd_pow_i<(D::d1 + F) & 3>(k, acc[3], r);
    }
}

template <int MU, bool FWD, bool FIRST, bool NEG>
__device__ __forceinline__ void x2_compute(const K2 &k, const float4 (&w)[8], const float4 &qh, const float4 &ql,
                                           cdd2 (&acc)[4])
{
    using D = X2Dir<MU, FWD>;
    cdd2 s[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        s[t].re = {make_float2(w[2 * t].x, w[2 * t].y), make_float2(w[2 * t + 1].x, w[2 * t + 1].y)};
        s[t].im = {make_float2(w[2 * t].z, w[2 * t].w), make_float2(w[2 * t + 1].z, w[2 * t + 1].w)};
    }
    // NEG: h_t = -s_t + i^c s_pi = -(s_t + i^{c+2} s_pi); the sign moves to the rebuild
    constexpr int F = NEG ? 2 : 0;
    const cdd2 h0 = cadd_pow_i<(D::c0 + F) & 3>(k, s[0], s[D::pi0]);
    const cdd2 h1 = cadd_pow_i<(D::c1 + F) & 3>(k, s[1], s[D::pi1]);
    const Link2 U = link2(qh, ql);
    // r_t = U h_t, each added into its upper spin and its lower partner at once
    // (rho maps the lower spins to r0 / r1), so only one r is live at a time
    x2_rebuild<0, D, F, FIRST>(k, su2_x2<FWD>(k, U, h0), acc);
    x2_rebuild<1, D, F, FIRST>(k, su2_x2<FWD>(k, U, h1), acc);
}

template <int MU, bool FWD, bool FIRST, bool NEG>
__device__ __forceinline__ void x2_term(const HopArgs &a, const K2 &k, int site_link, int link_par, int j_nb,
                                        cdd2 (&acc)[4])
{
    const float4 *sp = (const float4 *)a.in;
    float4 w[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) w[v] = __ldg(sp + vec_index(j_nb, v, 8));
    const size_t slot = (size_t)(link_par * 4 + MU) * a.g.nblk_g + (site_link >> 5);
    const float4 *qp = (const float4 *)a.gauge;
    const float4 qh = __ldg(qp + (slot * 2 + 0) * 32 + (site_link & 31));
    const float4 ql = __ldg(qp + (slot * 2 + 1) * 32 + (site_link & 31));
    x2_compute<MU, FWD, FIRST, NEG>(k, w, qh, ql, acc);
}

template <int MU, bool FIRST, bool NEG>
__device__ __forceinline__ void x2_dir(const HopArgs &a, const K2 &k, int i, int rr, const SiteNb &nb, cdd2 (&acc)[4])
{
    const int l = a.g.lrhs;
    x2_term<MU, true, FIRST, NEG>(a, k, i, a.p, (nb.fwd[MU] << l) + rr, acc);
    x2_term<MU, false, false, NEG>(a, k, nb.bwd[MU], 1 - a.p, (nb.bwd[MU] << l) + rr, acc);
}

// the site's epilogue: doublets back to values, then the shared epilogue
template <bool CLOV = false>
__device__ __forceinline__ void x2_epilogue(const HopArgs &a, int j, const cdd2 (&acc)[4], dd al, dd be, dd bu,
                                            SqAcc<dd> &red)
{
    cpx<dd> o[4][2];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        o[t][0] = {dd(acc[t].re.h.x, acc[t].re.l.x), dd(acc[t].im.h.x, acc[t].im.l.x)};
        o[t][1] = {dd(acc[t].re.h.y, acc[t].re.l.y), dd(acc[t].im.h.y, acc[t].im.l.y)};
    }
    hop_epilogue<kF64, CLOV>(a, j, o, al, be, bu, red);
}


// ---------------------------------------------------------------- binary16 projection
// h = s + i^C y on a packed (colour 0, colour 1) word pair (re, im)
template <int C>
__device__ __forceinline__ void h2_project(__half2 sre, __half2 sim, __half2 yre, __half2 yim, __half2 &hre,
                                           __half2 &him)
{
    if constexpr (C == 0) {
        hre = __hadd2(sre, yre);
        him = __hadd2(sim, yim);
    } else if constexpr (C == 1) {
        hre = __hsub2(sre, yim);
        him = __hadd2(sim, yre);
    } else if constexpr (C == 2) {
        hre = __hsub2(sre, yre);
        him = __hsub2(sim, yim);
    } else {
        hre = __hadd2(sre, yim);
        him = __hsub2(sim, yre);
    }
}

__device__ __forceinline__ __half2 as_h2(uint32_t u) { return *reinterpret_cast<const __half2 *>(&u); }

// acc (+)= i^C sc z
template <int C, bool FIRST>
__device__ __forceinline__ void acc_scaled(cpx<float> &acc, const cpx<float> &z, float sc)
{
    if constexpr (FIRST) {
        if constexpr (C == 0) acc = {sc * z.re, sc * z.im};
        else if constexpr (C == 1) acc = {-sc * z.im, sc * z.re};
        else if constexpr (C == 2) acc = {-sc * z.re, -sc * z.im};
        else acc = {sc * z.im, -sc * z.re};
    } else {
        if constexpr (C == 0) acc = {__fmaf_rn(sc, z.re, acc.re), __fmaf_rn(sc, z.im, acc.im)};
        else if constexpr (C == 1) acc = {__fmaf_rn(-sc, z.im, acc.re), __fmaf_rn(sc, z.re, acc.im)};
        else if constexpr (C == 2) acc = {__fmaf_rn(-sc, z.re, acc.re), __fmaf_rn(-sc, z.im, acc.im)};
        else acc = {__fmaf_rn(sc, z.im, acc.re), __fmaf_rn(-sc, z.re, acc.im)};
    }
}

// One direction's arithmetic from the neighbour's two packed words w0, w1, its
// scale sc and the link q (binary16, widened): acc (+)= (1 -/+ g_mu) U psi
// (FWD: U_mu(x), else U_mu(x - mu)^+).  NEG: the input's upper spins are
// negated (g5 in); as in the paired kernels the sign moves from the
// projection to the rebuild.
template <int MU, bool FWD, bool FIRST, bool NEG>
__device__ __forceinline__ void h16_compute(const uint4 &w0, const uint4 &w1, float sc, const float (&q)[4],
                                            cpx<float> (&acc)[4][2])
{
    using D = X2Dir<MU, FWD>;
    constexpr int F = NEG ? 2 : 0;
    // spin t: word 2t = (c0.re, c1.re), word 2t+1 = (c0.im, c1.im)
    const uint32_t u[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
    __half2 h0re, h0im, h1re, h1im;
    h2_project<(D::c0 + F) & 3>(as_h2(u[0]), as_h2(u[1]), as_h2(u[2 * D::pi0]), as_h2(u[2 * D::pi0 + 1]), h0re, h0im);
    h2_project<(D::c1 + F) & 3>(as_h2(u[2]), as_h2(u[3]), as_h2(u[2 * D::pi1]), as_h2(u[2 * D::pi1 + 1]), h1re, h1im);
    cpx<float> h[2][2];
    {
        const float2 r0 = __half22float2(h0re), i0 = __half22float2(h0im);
        const float2 r1 = __half22float2(h1re), i1 = __half22float2(h1im);
        h[0][0] = {r0.x, i0.x};
        h[0][1] = {r0.y, i0.y};
        h[1][0] = {r1.x, i1.x};
        h[1][1] = {r1.y, i1.y};
    }
    cpx<float> r[2][2];
    su2_mul<!FWD>(q, h[0], r[0]);
    su2_mul<!FWD>(q, h[1], r[1]);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        acc_scaled<F, FIRST>(acc[0][c], r[0][c], sc);
        acc_scaled<F, FIRST>(acc[1][c], r[1][c], sc);
        acc_scaled<(D::d0 + F) & 3, FIRST>(acc[2][c], r[D::rho0][c], sc);
        acc_scaled<(D::d1 + F) & 3, FIRST>(acc[3][c], r[D::rho1][c], sc);
    }
}

} // namespace hr
