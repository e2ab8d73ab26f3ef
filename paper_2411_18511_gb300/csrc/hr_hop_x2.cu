// hr_hop_x2.cu -- the paired hops (variants 10-13) on packed f32x2 FMAs:
// fundamental double-float with the two colours in the lanes, operands from
// registers (10, 12) or staged by cp.async one direction ahead (11, 13; 12 and
// 13 capped at 96 registers); adjoint double-float with (re, im) in the lanes
// (10, and 11 staged for quaternion links); FP32 arithmetic for FP32 / FP16
// storage (10, 11).
#include <algorithm>
#include <cstdlib>

#include "hr_hop_fam.h"
#include "hr_hop_x2.cuh"

using namespace hr;

namespace {

// Staged form: direction K+1's spinor and link are copied with cp.async into
// this thread's shared-memory slots while direction K is computed from the
// other buffer (as variant 1, with the paired arithmetic's half-size code).
template <int K, bool NEG>
__device__ __forceinline__ void x2_stage_step(const HopArgs &a, const K2 &k, int i, int rr, const SiteNb &nb,
                                              uint4 *b0, uint4 *b1, int bd, cdd2 (&acc)[4])
{
    uint4 *cur = (K & 1) ? b1 : b0;
    uint4 *nxt = (K & 1) ? b0 : b1;
    if constexpr (K < 7) {
        stage_issue<K + 1, kRepFund, kF64>(a, i, rr, nb, nxt, bd);
        cp_async_commit();
        cp_async_wait<1>();
    } else {
        cp_async_wait<0>();
    }
    float4 w[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) w[v] = *reinterpret_cast<const float4 *>(cur + v * bd);
    const float4 qh = *reinterpret_cast<const float4 *>(cur + 8 * bd);
    const float4 ql = *reinterpret_cast<const float4 *>(cur + 9 * bd);
    x2_compute<(K >> 1), (K & 1) == 0, K == 0, NEG>(k, w, qh, ql, acc);
}

template <int G5IN, bool CLOV = false>
__device__ __forceinline__ void x2s_body(const HopArgs &a)
{
    using S = Stage<kRepFund, kF64>;
    static_assert(S::NSLOT == 10, "8 spinor + 2 link vectors per direction");
    constexpr bool NEG = G5IN != 0;
    extern __shared__ uint4 x2_stage_mem[];
    if ((a.gate && *a.gate == 0.0) || (a.done && *a.done != 0.0)) return;
    const K2 k = make_k2(a.unit, a.nil);
    const Geom &g = a.g;
    const int nv = g.vh << g.lrhs;
    const int stride = gridDim.x * blockDim.x;
    const int bd = blockDim.x;
    uint4 *b0 = x2_stage_mem + threadIdx.x;
    uint4 *b1 = x2_stage_mem + S::NSLOT * bd + threadIdx.x;
    const dd be = Real<dd>::from_coef(a.beta);
    const dd bu = a.g5_out ? -be : be;
    const dd al = Real<dd>::from_coef(a.alpha);
    SqAcc<dd> red;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nv; j += stride) {
        const int i = j >> g.lrhs, rr = j & (g.nrhs - 1);
        SiteNb nb;
        site_neighbours(g, i, a.p, nb);
        stage_issue<0, kRepFund, kF64>(a, i, rr, nb, b0, bd);
        cp_async_commit();
        cdd2 acc[4];
        x2_stage_step<0, NEG>(a, k, i, rr, nb, b0, b1, bd, acc);
        x2_stage_step<1, NEG>(a, k, i, rr, nb, b0, b1, bd, acc);
        x2_stage_step<2, NEG>(a, k, i, rr, nb, b0, b1, bd, acc);
        x2_stage_step<3, NEG>(a, k, i, rr, nb, b0, b1, bd, acc);
        x2_stage_step<4, NEG>(a, k, i, rr, nb, b0, b1, bd, acc);
        x2_stage_step<5, NEG>(a, k, i, rr, nb, b0, b1, bd, acc);
        x2_stage_step<6, NEG>(a, k, i, rr, nb, b0, b1, bd, acc);
        x2_stage_step<7, NEG>(a, k, i, rr, nb, b0, b1, bd, acc);
        x2_epilogue<CLOV>(a, j, acc, al, be, bu, red);
    }
    if (a.fin) {
        __shared__ double smem[32 * 32];
        __shared__ double sums[32];
        if (grid_reduce(red, g.nrhs, a.red, sums, smem)) finish_reduction(a.fin, sums, g.nrhs, a.scal);
    }
}

template <int G5IN>
__device__ __forceinline__ void x2_body(const HopArgs &a)
{
    using T = dd;
    constexpr bool NEG = G5IN != 0;
    if ((a.gate && *a.gate == 0.0) || (a.done && *a.done != 0.0)) return;
    const K2 k = make_k2(a.unit, a.nil);
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
        epilogue_prefetch<2, kF64>(a, j);
        cdd2 acc[4];
        x2_dir<0, true, NEG>(a, k, i, rr, nb, acc);
        x2_dir<1, false, NEG>(a, k, i, rr, nb, acc);
        x2_dir<2, false, NEG>(a, k, i, rr, nb, acc);
        x2_dir<3, false, NEG>(a, k, i, rr, nb, acc);
        x2_epilogue(a, j, acc, al, be, bu, red);
    }
    if (a.fin) {
        __shared__ double smem[32 * 32];
        __shared__ double sums[32];
        if (grid_reduce(red, g.nrhs, a.red, sums, smem)) finish_reduction(a.fin, sums, g.nrhs, a.scal);
    }
}

// registers as the compiler likes (about 100 / 128), or capped at 96: five
// 128-thread blocks per SM (the staged form's 40 KB of slots each still fit)
template <int G5IN> __global__ void __launch_bounds__(256) k_hop_x2(HopArgs a) { x2_body<G5IN>(a); }
template <int G5IN> __global__ void __maxnreg__(96) k_hop_x2_r96(HopArgs a) { x2_body<G5IN>(a); }
template <int G5IN> __global__ void __launch_bounds__(256) k_hop_x2s(HopArgs a) { x2s_body<G5IN>(a); }
template <int G5IN> __global__ void __launch_bounds__(256) k_hop_x2s_clov(HopArgs a) { x2s_body<G5IN, true>(a); }
template <int G5IN> __global__ void __maxnreg__(96) k_hop_x2s_r96(HopArgs a) { x2s_body<G5IN>(a); }

// ---------------------------------------------------------------- FP32 / FP16 storage
// The same pairing for the FP32-arithmetic hops: the FP32 and FP16 layouts are
// colour-paired too (per spin (c0.re, c1.re, c0.im, c1.im)), a vector gives
// lane pairs at once, and each colour-product output is one packed multiply
// and three packed FMAs.  Results agree with the scalar kernels to rounding
// (their FMA contraction is the compiler's), not bit for bit.

struct cf2 {
    float2 re, im; // a colour doublet of complex numbers
};

template <int S> __device__ __forceinline__ float2 fadd_s(const K2 &k, float2 a, float2 b)
{
    return __ffma2_rn(b, S > 0 ? k.one : k.mone, a); // a + S b
}
// x + i^C y
template <int C> __device__ __forceinline__ cf2 fadd_pow_i(const K2 &k, const cf2 &x, const cf2 &y)
{
    if constexpr (C == 0) return {fadd_s<1>(k, x.re, y.re), fadd_s<1>(k, x.im, y.im)};
    else if constexpr (C == 1) return {fadd_s<-1>(k, x.re, y.im), fadd_s<1>(k, x.im, y.re)};
    else if constexpr (C == 2) return {fadd_s<-1>(k, x.re, y.re), fadd_s<-1>(k, x.im, y.im)};
    else return {fadd_s<1>(k, x.re, y.im), fadd_s<-1>(k, x.im, y.re)};
}
// i^C y
template <int C> __device__ __forceinline__ cf2 fpow_i(const K2 &k, const cf2 &y)
{
    const auto neg = [&](float2 v) { return __ffma2_rn(v, k.mone, k.zero); };
    if constexpr (C == 0) return y;
    else if constexpr (C == 1) return {neg(y.im), y.re};
    else if constexpr (C == 2) return {neg(y.re), neg(y.im)};
    else return {y.im, neg(y.re)};
}

// link coefficient pairs (see Link2) and their negations
struct Link2f {
    float2 c0, c1, c2, c3, n1, n2, n3;
};
__device__ __forceinline__ Link2f link2f(float a0, float a1, float a2, float a3)
{
    Link2f L;
    L.c0 = make_float2(a0, a0);
    L.c1 = make_float2(a1, a1);
    L.c2 = make_float2(a2, -a2);
    L.c3 = make_float2(a3, -a3);
    L.n1 = make_float2(-a1, -a1);
    L.n2 = make_float2(-a2, a2);
    L.n3 = make_float2(-a3, a3);
    return L;
}
// r = U h (FWD) or U^+ h: re = C0 hr -/+ C3 hi +/- C2 sr -/+ C1 si,
// im = C0 hi +/- C3 hr +/- C2 si +/- C1 sr (s = swap(h); upper signs forward)
template <bool FWD> __device__ __forceinline__ cf2 su2_f2(const K2 &k, const Link2f &U, const cf2 &h)
{
    const float2 sr = swap2(h.re), si = swap2(h.im);
    const float2 p3 = FWD ? U.c3 : U.n3, m3 = FWD ? U.n3 : U.c3;
    const float2 p2 = FWD ? U.c2 : U.n2, p1 = FWD ? U.c1 : U.n1, m1 = FWD ? U.n1 : U.c1;
    cf2 r;
    r.re = __ffma2_rn(U.c0, h.re, k.zero);
    r.re = __ffma2_rn(m3, h.im, r.re);
    r.re = __ffma2_rn(p2, sr, r.re);
    r.re = __ffma2_rn(m1, si, r.re);
    r.im = __ffma2_rn(U.c0, h.im, k.zero);
    r.im = __ffma2_rn(p3, h.re, r.im);
    r.im = __ffma2_rn(p2, si, r.im);
    r.im = __ffma2_rn(p1, sr, r.im);
    return r;
}

template <int T, class D, int F, bool FIRST>
__device__ __forceinline__ void f2_rebuild(const K2 &k, const cf2 &r, cf2 (&acc)[4])
{
    if constexpr (FIRST) acc[T] = fpow_i<F>(k, r);
    else acc[T] = fadd_pow_i<F>(k, acc[T], r);
    if constexpr (D::rho0 == T) {
        if constexpr (FIRST) acc[2] = fpow_i<(D::d0 + F) & 3>(k, r);
        else acc[2] = fadd_pow_i<(D::d0 + F) & 3>(k, acc[2], r);
    }
    if constexpr (D::rho1 == T) {
        if constexpr (FIRST) acc[3] = fpow_i<(D::d1 + F) & 3>(k, r);
        else acc[3] = fadd_pow_i<(D::d1 + F) & 3>(k, acc[3], r);
    }
}

// one direction from the site's 8 packed reals (spin t: re pair, im pair) and
// the link scaled by sc (binary16: the neighbour's scale rides on the link)
template <int MU, bool FWD, bool FIRST, bool NEG>
__device__ __forceinline__ void f2_compute(const K2 &k, const float2 (&sv)[8], float a0, float a1, float a2, float a3,
                                           cf2 (&acc)[4])
{
    using D = X2Dir<MU, FWD>;
    cf2 s[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) s[t] = {sv[2 * t], sv[2 * t + 1]};
    constexpr int F = NEG ? 2 : 0;
    const cf2 h0 = fadd_pow_i<(D::c0 + F) & 3>(k, s[0], s[D::pi0]);
    const cf2 h1 = fadd_pow_i<(D::c1 + F) & 3>(k, s[1], s[D::pi1]);
    const Link2f U = link2f(a0, a1, a2, a3);
    f2_rebuild<0, D, F, FIRST>(k, su2_f2<FWD>(k, U, h0), acc);
    f2_rebuild<1, D, F, FIRST>(k, su2_f2<FWD>(k, U, h1), acc);
}

// the packed reals of a site as 8 lane pairs, and its binary16 scale
template <int PREC>
__device__ __forceinline__ void f2_load_site(const HopArgs &a, int j, float2 (&sv)[8], float &sc)
{
    if constexpr (PREC == kF32) {
        const float4 *p = (const float4 *)a.in;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const float4 w = __ldg(p + vec_index(j, v, 4));
            sv[2 * v] = make_float2(w.x, w.y);
            sv[2 * v + 1] = make_float2(w.z, w.w);
        }
        sc = 1.f;
    } else {
        const uint4 *p = (const uint4 *)a.in;
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            const uint4 w = __ldg(p + vec_index(j, v, 2));
            const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) sv[4 * v + q] = __half22float2(*reinterpret_cast<const __half2 *>(&u[q]));
        }
        sc = __ldg((const float *)((const char *)a.in + SpinorLayout<2, kF16>::data_bytes(a.g.nblk_s)) + j);
    }
}

template <int MU, bool FWD, bool FIRST, bool NEG, int PREC>
__device__ __forceinline__ void f2_term(const HopArgs &a, const K2 &k, int site_link, int link_par, int j_nb,
                                        cf2 (&acc)[4])
{
    float2 sv[8];
    float sc;
    f2_load_site<PREC>(a, j_nb, sv, sc);
    float q[4];
    load_quat<PREC>(a.gauge, a.g.nblk_g, link_par, MU, site_link, q);
    if constexpr (PREC == kF16) {
#pragma unroll
        for (int c = 0; c < 4; ++c) q[c] *= sc;
    }
    f2_compute<MU, FWD, FIRST, NEG>(k, sv, q[0], q[1], q[2], q[3], acc);
}

template <int MU, bool FIRST, bool NEG, int PREC>
__device__ __forceinline__ void f2_dir(const HopArgs &a, const K2 &k, int i, int rr, const SiteNb &nb, cf2 (&acc)[4])
{
    const int l = a.g.lrhs;
    f2_term<MU, true, FIRST, NEG, PREC>(a, k, i, a.p, (nb.fwd[MU] << l) + rr, acc);
    f2_term<MU, false, false, NEG, PREC>(a, k, nb.bwd[MU], 1 - a.p, (nb.bwd[MU] << l) + rr, acc);
}

template <int PREC, int G5IN>
__device__ __forceinline__ void f2_body(const HopArgs &a)
{
    constexpr bool NEG = G5IN != 0;
    if ((a.gate && *a.gate == 0.0) || (a.done && *a.done != 0.0)) return;
    const K2 k = make_k2(a.unit, a.nil);
    const Geom &g = a.g;
    const int nv = g.vh << g.lrhs;
    const int stride = gridDim.x * blockDim.x;
    const float be = a.beta.h;
    const float bu = a.g5_out ? -be : be;
    const float al = a.alpha.h;
    SqAcc<float> red;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nv; j += stride) {
        const int i = j >> g.lrhs, rr = j & (g.nrhs - 1);
        SiteNb nb;
        site_neighbours(g, i, a.p, nb);
        cf2 acc[4];
        f2_dir<0, true, NEG, PREC>(a, k, i, rr, nb, acc);
        f2_dir<1, false, NEG, PREC>(a, k, i, rr, nb, acc);
        f2_dir<2, false, NEG, PREC>(a, k, i, rr, nb, acc);
        f2_dir<3, false, NEG, PREC>(a, k, i, rr, nb, acc);
        cpx<float> o[4][2];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            o[t][0] = {acc[t].re.x, acc[t].im.x};
            o[t][1] = {acc[t].re.y, acc[t].im.y};
        }
        hop_epilogue<PREC>(a, j, o, al, be, bu, red);
    }
    if (a.fin) {
        __shared__ double smem[32 * 32];
        __shared__ double sums[32];
        if (grid_reduce(red, g.nrhs, a.red, sums, smem)) finish_reduction(a.fin, sums, g.nrhs, a.scal);
    }
}

// staged form: direction K+1's operands copied by cp.async while K is computed
template <int K, bool NEG, int PREC>
__device__ __forceinline__ void f2_stage_step(const HopArgs &a, const K2 &k, int i, int rr, const SiteNb &nb,
                                              uint4 *b0, uint4 *b1, int bd, cf2 (&acc)[4])
{
    using S = Stage<kRepFund, PREC>;
    uint4 *cur = (K & 1) ? b1 : b0;
    uint4 *nxt = (K & 1) ? b0 : b1;
    if constexpr (K < 7) {
        stage_issue<K + 1, kRepFund, PREC>(a, i, rr, nb, nxt, bd);
        cp_async_commit();
        cp_async_wait<1>();
    } else {
        cp_async_wait<0>();
    }
    float2 sv[8];
    float q[4];
    if constexpr (PREC == kF32) {
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const float4 w = *reinterpret_cast<const float4 *>(cur + v * bd);
            sv[2 * v] = make_float2(w.x, w.y);
            sv[2 * v + 1] = make_float2(w.z, w.w);
        }
        const float4 qv = *reinterpret_cast<const float4 *>(cur + S::NV * bd);
        q[0] = qv.x; q[1] = qv.y; q[2] = qv.z; q[3] = qv.w;
    } else {
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            const uint4 w = cur[v * bd];
            const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int c = 0; c < 4; ++c) sv[4 * v + c] = __half22float2(*reinterpret_cast<const __half2 *>(&u[c]));
        }
        // the link slot holds 8 bytes (cp.async of a uint2), the scale slot 4
        const uint2 qw = *reinterpret_cast<const uint2 *>(cur + S::NV * bd);
        const float2 q01 = __half22float2(*reinterpret_cast<const __half2 *>(&qw.x));
        const float2 q23 = __half22float2(*reinterpret_cast<const __half2 *>(&qw.y));
        const float sc = *reinterpret_cast<const float *>(cur + (S::NV + S::NQ) * bd);
        q[0] = q01.x * sc; q[1] = q01.y * sc; q[2] = q23.x * sc; q[3] = q23.y * sc;
    }
    f2_compute<(K >> 1), (K & 1) == 0, K == 0, NEG>(k, sv, q[0], q[1], q[2], q[3], acc);
}

template <int PREC, int G5IN>
__device__ __forceinline__ void f2s_body(const HopArgs &a)
{
    using S = Stage<kRepFund, PREC>;
    constexpr bool NEG = G5IN != 0;
    extern __shared__ uint4 f2_stage_mem[];
    if ((a.gate && *a.gate == 0.0) || (a.done && *a.done != 0.0)) return;
    const K2 k = make_k2(a.unit, a.nil);
    const Geom &g = a.g;
    const int nv = g.vh << g.lrhs;
    const int stride = gridDim.x * blockDim.x;
    const int bd = blockDim.x;
    uint4 *b0 = f2_stage_mem + threadIdx.x;
    uint4 *b1 = f2_stage_mem + S::NSLOT * bd + threadIdx.x;
    const float be = a.beta.h;
    const float bu = a.g5_out ? -be : be;
    const float al = a.alpha.h;
    SqAcc<float> red;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nv; j += stride) {
        const int i = j >> g.lrhs, rr = j & (g.nrhs - 1);
        SiteNb nb;
        site_neighbours(g, i, a.p, nb);
        stage_issue<0, kRepFund, PREC>(a, i, rr, nb, b0, bd);
        cp_async_commit();
        cf2 acc[4];
        f2_stage_step<0, NEG, PREC>(a, k, i, rr, nb, b0, b1, bd, acc);
        f2_stage_step<1, NEG, PREC>(a, k, i, rr, nb, b0, b1, bd, acc);
        f2_stage_step<2, NEG, PREC>(a, k, i, rr, nb, b0, b1, bd, acc);
        f2_stage_step<3, NEG, PREC>(a, k, i, rr, nb, b0, b1, bd, acc);
        f2_stage_step<4, NEG, PREC>(a, k, i, rr, nb, b0, b1, bd, acc);
        f2_stage_step<5, NEG, PREC>(a, k, i, rr, nb, b0, b1, bd, acc);
        f2_stage_step<6, NEG, PREC>(a, k, i, rr, nb, b0, b1, bd, acc);
        f2_stage_step<7, NEG, PREC>(a, k, i, rr, nb, b0, b1, bd, acc);
        cpx<float> o[4][2];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            o[t][0] = {acc[t].re.x, acc[t].im.x};
            o[t][1] = {acc[t].re.y, acc[t].im.y};
        }
        hop_epilogue<PREC>(a, j, o, al, be, bu, red);
    }
    if (a.fin) {
        __shared__ double smem[32 * 32];
        __shared__ double sums[32];
        if (grid_reduce(red, g.nrhs, a.red, sums, smem)) finish_reduction(a.fin, sums, g.nrhs, a.scal);
    }
}

template <int PREC, int G5IN> __global__ void __launch_bounds__(256) k_hop_f2(HopArgs a) { f2_body<PREC, G5IN>(a); }
template <int PREC, int G5IN> __global__ void __launch_bounds__(256) k_hop_f2s(HopArgs a) { f2s_body<PREC, G5IN>(a); }

// ---------------------------------------------------------------- adjoint FP64, (re, im) lanes
// With three colours the lanes are the real and imaginary parts of one complex
// double-float: the FP64 layout for three colours already stores (re.h, im.h,
// re.l, im.l), and the adjoint links are real, so a colour product scales both
// lanes by one link entry (a duplicated lane pair).  A factor +-i swaps the
// lanes with a (-1, 1) or (1, -1) sign pattern.  Sums in the scalar kernel's
// order: bit-identical results, as for the fundamental pairing.

// x + i^C y for complex (re, im) lane pairs
template <int C> __device__ __forceinline__ dd2 cx_add_pow_i(const K2 &k, const dd2 &x, const dd2 &y)
{
    if constexpr (C == 0) return add2v(k, x, y, k.one);
    else if constexpr (C == 2) return add2v(k, x, y, k.mone);
    else if constexpr (C == 1) return add2v(k, x, swap2(y), k.mp); // (x.re - y.im, x.im + y.re)
    else return add2v(k, x, swap2(y), k.pm);                       // (x.re + y.im, x.im - y.re)
}
// i^C y
template <int C> __device__ __forceinline__ dd2 cx_pow_i(const K2 &k, const dd2 &y)
{
    if constexpr (C == 0) return y;
    else if constexpr (C == 2) return neg2(k, y);
    else {
        const float2 sg = C == 1 ? k.mp : k.pm;
        const dd2 t = swap2(y);
        return {__ffma2_rn(t.h, sg, k.zero), __ffma2_rn(t.l, sg, k.zero)};
    }
}

// the value sg c x of a product in its prod2 form, sg a lane pair of powers of
// two (exact); nsg = -sg
__device__ __forceinline__ dd2 prod2_scaled(const K2 &k, const prod2 &p, float2 nsg, float2 sg)
{
    return {__ffma2_rn(p.P, nsg, k.zero), __ffma2_rn(p.L, sg, k.zero)};
}
// r + sg c x lane by lane for a product in its prod2 form (sg a power of two
// per lane, nsg = -sg): add2v on the exactly scaled product
__device__ __forceinline__ dd2 acc_prod2v(const K2 &k, const dd2 &r, const prod2 &p, float2 nsg, float2 sg)
{
    const float2 s = __ffma2_rn(p.P, nsg, r.h);
    const float2 w = __ffma2_rn(s, k.mone, r.h);
    const float2 t = __ffma2_rn(w, k.one, s);
    const float2 da = __ffma2_rn(t, k.mone, r.h);
    const float2 db = __ffma2_rn(p.P, nsg, w);
    const float2 e = __ffma2_rn(da, k.one, db);
    const float2 lo = __ffma2_rn(p.L, sg, r.l);
    return {s, __ffma2_rn(e, k.one, lo)};
}
__device__ __forceinline__ dd2 dup2(const dd &x) { return {make_float2(x.h, x.h), make_float2(x.l, x.l)}; }
__device__ __forceinline__ dd lane_x(const dd2 &v) { return dd(v.h.x, v.l.x); }
__device__ __forceinline__ dd lane_y(const dd2 &v) { return dd(v.h.y, v.l.y); }

// R(q) from the packed quaternion (hi parts qh, lo parts ql) with the scalar
// quat_to_adj's operations, two entries per f32x2 instruction where the
// entries pair up: the squares (a0^2, a1^2), (a2^2, a3^2); (a0^2 - a2^2,
// a1^2 + a3^2) for w; the diagonal pair (R11, R22); the products a1 (a2, a3)
// and a0 (a3, a2), which give (R01, R02) and (R10, R20); (R12, R21).  Each
// lane does the scalar operation on the same operands, so R is bit-identical
// to the scalar rebuild's.
__device__ __forceinline__ void quat_to_adj_x2(const K2 &k, const float4 &qh, const float4 &ql, dd (&R)[3][3])
{
    const bool neg = sign_bit(qh.x);
    const float s2 = neg ? -2.f : 2.f;
    const dd2 q01 = {make_float2(qh.x, qh.y), make_float2(ql.x, ql.y)};
    const dd2 q23 = {make_float2(qh.z, qh.w), make_float2(ql.z, ql.w)};
    const dd2 q32 = {make_float2(qh.w, qh.z), make_float2(ql.w, ql.z)};
    const prod2 p01 = mul2(k, q01, make_float2(-qh.x, -qh.y), q01);
    const prod2 p23 = mul2(k, q23, make_float2(-qh.z, -qh.w), q23);
    const dd2 s01 = prod2_scaled(k, p01, k.mone, k.one), s23 = prod2_scaled(k, p23, k.mone, k.one);
    const dd2 d = add2v(k, s01, s23, k.mp); // (a0^2 - a2^2, a1^2 + a3^2)
    dd w = lane_x(d) - lane_y(d);
    if (neg) w = -w;
    R[0][0] = w + scale_pow2(lane_y(s01), s2);
    const dd2 r12 = add2v(k, dup2(w), s23, make_float2(s2, s2));
    R[1][1] = lane_x(r12);
    R[2][2] = lane_y(r12);
    const dd a0(qh.x, ql.x), a1(qh.y, ql.y), a2(qh.z, ql.z), a3(qh.w, ql.w);
    const prod2 x = mul2(k, dup2(a1), make_float2(-a1.h, -a1.h), q23); // a1 (a2, a3)
    const prod2 y = mul2(k, dup2(a0), make_float2(-a0.h, -a0.h), q32); // a0 (a3, a2)
    const dd2 xs = prod2_scaled(k, x, make_float2(-s2, -s2), make_float2(s2, s2));
    const dd2 u = acc_prod2v(k, xs, y, make_float2(-s2, s2), make_float2(s2, -s2));
    const dd2 v = acc_prod2v(k, xs, y, make_float2(s2, -s2), make_float2(-s2, s2));
    R[0][1] = lane_x(u); R[0][2] = lane_y(u);
    R[1][0] = lane_x(v); R[2][0] = lane_y(v);
    const dd m23 = scale_pow2(a2 * a3, s2), m01 = a0 * a1;
    const dd2 t = add2v(k, dup2(m23), dup2(m01), make_float2(s2, -s2));
    R[1][2] = lane_x(t); R[2][1] = lane_y(t);
}

// r_t,b = sum_c M_bc h_t,c for both half-spinor components t at one output
// colour b, M = R (forward) or R^T (backward), in the scalar kernel's order
template <bool FWD, int B>
__device__ __forceinline__ void so3_row_x2(const K2 &k, const dd (&R)[3][3], const dd2 (&h)[2][3], dd2 (&r)[2])
{
    dd2 c[3];
    float2 n[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        const dd m = FWD ? R[B][e] : R[e][B];
        c[e] = {make_float2(m.h, m.h), make_float2(m.l, m.l)};
        n[e] = make_float2(-m.h, -m.h);
    }
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        r[t] = first_prod2<1>(k, mul2(k, c[0], n[0], h[t][0]));
        r[t] = acc_prod2<1>(k, r[t], mul2(k, c[1], n[1], h[t][1]));
        r[t] = acc_prod2<1>(k, r[t], mul2(k, c[2], n[2], h[t][2]));
    }
}

// acc_t,b (+)= i^F r_t and acc_{2+u},b (+)= i^{d_u + F} r_{rho_u} at colour b
template <class D, int F, bool FIRST, int B>
__device__ __forceinline__ void x2a_rebuild(const K2 &k, const dd2 (&r)[2], dd2 (&acc)[4][3])
{
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        if constexpr (FIRST) acc[t][B] = cx_pow_i<F>(k, r[t]);
        else acc[t][B] = cx_add_pow_i<F>(k, acc[t][B], r[t]);
    }
    if constexpr (FIRST) {
        acc[2][B] = cx_pow_i<(D::d0 + F) & 3>(k, r[D::rho0]);
        acc[3][B] = cx_pow_i<(D::d1 + F) & 3>(k, r[D::rho1]);
    } else {
        acc[2][B] = cx_add_pow_i<(D::d0 + F) & 3>(k, acc[2][B], r[D::rho0]);
        acc[3][B] = cx_add_pow_i<(D::d1 + F) & 3>(k, acc[3][B], r[D::rho1]);
    }
}

template <int MU, bool FWD, bool FIRST, bool NEG>
__device__ __forceinline__ void x2a_compute(const K2 &k, const float4 (&w)[12], const dd (&R)[3][3], dd2 (&acc)[4][3])
{
    using D = X2Dir<MU, FWD>;
    constexpr int F = NEG ? 2 : 0;
    dd2 h[2][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const auto sv = [&](int t) -> dd2 {
            const float4 v = w[3 * t + c];
            return {make_float2(v.x, v.y), make_float2(v.z, v.w)};
        };
        h[0][c] = cx_add_pow_i<(D::c0 + F) & 3>(k, sv(0), sv(D::pi0));
        h[1][c] = cx_add_pow_i<(D::c1 + F) & 3>(k, sv(1), sv(D::pi1));
    }
    dd2 r[2];
    so3_row_x2<FWD, 0>(k, R, h, r);
    x2a_rebuild<D, F, FIRST, 0>(k, r, acc);
    so3_row_x2<FWD, 1>(k, R, h, r);
    x2a_rebuild<D, F, FIRST, 1>(k, r, acc);
    so3_row_x2<FWD, 2>(k, R, h, r);
    x2a_rebuild<D, F, FIRST, 2>(k, r, acc);
}

template <int REP>
__device__ __forceinline__ void x2a_link(const HopArgs &a, const K2 &k, int link_par, int mu, int site_link,
                                         dd (&R)[3][3])
{
    if constexpr (REP == kRepAdj) {
        const size_t slot = (size_t)(link_par * 4 + mu) * a.g.nblk_g + (site_link >> 5);
        const float4 *q = (const float4 *)a.gauge + slot * 64 + (site_link & 31);
        quat_to_adj_x2(k, __ldg(q), __ldg(q + 32), R);
    } else {
        load_mat<kF64>(a.gauge, a.g.nblk_g, link_par, mu, site_link, R);
    }
}

template <int MU, bool FWD, bool FIRST, bool NEG, int REP>
__device__ __forceinline__ void x2a_term(const HopArgs &a, const K2 &k, int site_link, int link_par, int j_nb,
                                         dd2 (&acc)[4][3])
{
    const float4 *sp = (const float4 *)a.in;
    float4 w[12];
#pragma unroll
    for (int v = 0; v < 12; ++v) w[v] = __ldg(sp + vec_index(j_nb, v, 12));
    dd R[3][3];
    x2a_link<REP>(a, k, link_par, MU, site_link, R);
    x2a_compute<MU, FWD, FIRST, NEG>(k, w, R, acc);
}

__device__ __forceinline__ void x2a_epilogue(const HopArgs &a, int j, const dd2 (&acc)[4][3], dd al, dd be, dd bu,
                                             SqAcc<dd> &red)
{
    cpx<dd> o[4][3];
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
        for (int c = 0; c < 3; ++c) o[t][c] = {dd(acc[t][c].h.x, acc[t][c].l.x), dd(acc[t][c].h.y, acc[t][c].l.y)};
    hop_epilogue<kF64>(a, j, o, al, be, bu, red);
}

template <int REP, int G5IN>
__device__ __forceinline__ void x2a_body(const HopArgs &a)
{
    constexpr bool NEG = G5IN != 0;
    if ((a.gate && *a.gate == 0.0) || (a.done && *a.done != 0.0)) return;
    const K2 k = make_k2(a.unit, a.nil);
    const Geom &g = a.g;
    const int nv = g.vh << g.lrhs;
    const int stride = gridDim.x * blockDim.x;
    const int l = g.lrhs;
    const dd be = Real<dd>::from_coef(a.beta);
    const dd bu = a.g5_out ? -be : be;
    const dd al = Real<dd>::from_coef(a.alpha);
    SqAcc<dd> red;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nv; j += stride) {
        const int i = j >> l, rr = j & (g.nrhs - 1);
        SiteNb nb;
        site_neighbours(g, i, a.p, nb);
        dd2 acc[4][3];
        x2a_term<0, true, true, NEG, REP>(a, k, i, a.p, (nb.fwd[0] << l) + rr, acc);
        x2a_term<0, false, false, NEG, REP>(a, k, nb.bwd[0], 1 - a.p, (nb.bwd[0] << l) + rr, acc);
        x2a_term<1, true, false, NEG, REP>(a, k, i, a.p, (nb.fwd[1] << l) + rr, acc);
        x2a_term<1, false, false, NEG, REP>(a, k, nb.bwd[1], 1 - a.p, (nb.bwd[1] << l) + rr, acc);
        x2a_term<2, true, false, NEG, REP>(a, k, i, a.p, (nb.fwd[2] << l) + rr, acc);
        x2a_term<2, false, false, NEG, REP>(a, k, nb.bwd[2], 1 - a.p, (nb.bwd[2] << l) + rr, acc);
        x2a_term<3, true, false, NEG, REP>(a, k, i, a.p, (nb.fwd[3] << l) + rr, acc);
        x2a_term<3, false, false, NEG, REP>(a, k, nb.bwd[3], 1 - a.p, (nb.bwd[3] << l) + rr, acc);
        x2a_epilogue(a, j, acc, al, be, bu, red);
    }
    if (a.fin) {
        __shared__ double smem[32 * 32];
        __shared__ double sums[32];
        if (grid_reduce(red, g.nrhs, a.red, sums, smem)) finish_reduction(a.fin, sums, g.nrhs, a.scal);
    }
}

// staged form (quaternion links): direction K+1's operands copied by cp.async while K is computed
template <int K, bool NEG>
__device__ __forceinline__ void x2a_stage_step(const HopArgs &a, const K2 &k, int i, int rr, const SiteNb &nb,
                                               uint4 *b0, uint4 *b1, int bd, dd2 (&acc)[4][3])
{
    uint4 *cur = (K & 1) ? b1 : b0;
    uint4 *nxt = (K & 1) ? b0 : b1;
    if constexpr (K < 7) {
        stage_issue<K + 1, kRepAdj, kF64>(a, i, rr, nb, nxt, bd);
        cp_async_commit();
        cp_async_wait<1>();
    } else {
        cp_async_wait<0>();
    }
    float4 w[12];
#pragma unroll
    for (int v = 0; v < 12; ++v) w[v] = *reinterpret_cast<const float4 *>(cur + v * bd);
    const float4 qh = *reinterpret_cast<const float4 *>(cur + 12 * bd);
    const float4 ql = *reinterpret_cast<const float4 *>(cur + 13 * bd);
    dd R[3][3];
    quat_to_adj_x2(k, qh, ql, R);
    x2a_compute<(K >> 1), (K & 1) == 0, K == 0, NEG>(k, w, R, acc);
}

template <int G5IN>
__device__ __forceinline__ void x2as_body(const HopArgs &a)
{
    using S = Stage<kRepAdj, kF64>;
    static_assert(S::NSLOT == 14, "12 spinor + 2 link vectors per direction");
    constexpr bool NEG = G5IN != 0;
    extern __shared__ uint4 x2a_stage_mem[];
    if ((a.gate && *a.gate == 0.0) || (a.done && *a.done != 0.0)) return;
    const K2 k = make_k2(a.unit, a.nil);
    const Geom &g = a.g;
    const int nv = g.vh << g.lrhs;
    const int stride = gridDim.x * blockDim.x;
    const int bd = blockDim.x;
    uint4 *b0 = x2a_stage_mem + threadIdx.x;
    uint4 *b1 = x2a_stage_mem + S::NSLOT * bd + threadIdx.x;
    const dd be = Real<dd>::from_coef(a.beta);
    const dd bu = a.g5_out ? -be : be;
    const dd al = Real<dd>::from_coef(a.alpha);
    SqAcc<dd> red;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nv; j += stride) {
        const int i = j >> g.lrhs, rr = j & (g.nrhs - 1);
        SiteNb nb;
        site_neighbours(g, i, a.p, nb);
        stage_issue<0, kRepAdj, kF64>(a, i, rr, nb, b0, bd);
        cp_async_commit();
        dd2 acc[4][3];
        x2a_stage_step<0, NEG>(a, k, i, rr, nb, b0, b1, bd, acc);
        x2a_stage_step<1, NEG>(a, k, i, rr, nb, b0, b1, bd, acc);
        x2a_stage_step<2, NEG>(a, k, i, rr, nb, b0, b1, bd, acc);
        x2a_stage_step<3, NEG>(a, k, i, rr, nb, b0, b1, bd, acc);
        x2a_stage_step<4, NEG>(a, k, i, rr, nb, b0, b1, bd, acc);
        x2a_stage_step<5, NEG>(a, k, i, rr, nb, b0, b1, bd, acc);
        x2a_stage_step<6, NEG>(a, k, i, rr, nb, b0, b1, bd, acc);
        x2a_stage_step<7, NEG>(a, k, i, rr, nb, b0, b1, bd, acc);
        x2a_epilogue(a, j, acc, al, be, bu, red);
    }
    if (a.fin) {
        __shared__ double smem[32 * 32];
        __shared__ double sums[32];
        if (grid_reduce(red, g.nrhs, a.red, sums, smem)) finish_reduction(a.fin, sums, g.nrhs, a.scal);
    }
}

template <int REP, int G5IN> __global__ void __maxnreg__(128) k_hop_x2a(HopArgs a) { x2a_body<REP, G5IN>(a); }
// the same with up to 168 registers: no spills (the 128-register form spills
// about 100 bytes a thread for the quaternion links), 12 warps an SM at
// blocks of 64, 128 or 192 threads
template <int REP, int G5IN> __global__ void __maxnreg__(168) k_hop_x2a_big(HopArgs a) { x2a_body<REP, G5IN>(a); }
template <int G5IN> __global__ void __launch_bounds__(256) k_hop_x2as(HopArgs a) { x2as_body<G5IN>(a); }

template <int REP, int PREC> struct Launch {
    static bool run(hr_ctx *ctx, const Geom &, const HopArgs &a, HopChoice c, int grid, cudaStream_t s,
                    hr_status &st)
    {
        if constexpr (REP == kRepFund && PREC == kF64) {
            using S = Stage<kRepFund, kF64>;
            static bool attr_set = false;
            if (!attr_set) {
                for (auto f : {k_hop_x2s<0>, k_hop_x2s<1>, k_hop_x2s_r96<0>, k_hop_x2s_r96<1>})
                    cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::smem_bytes(256));
                attr_set = true;
            }
            const size_t sm = S::smem_bytes(c.block);
            const bool g5 = a.g5_in != 0;
            switch (c.variant) {
            case kVarPairedStaged: (g5 ? k_hop_x2s<1> : k_hop_x2s<0>)<<<grid, c.block, sm, s>>>(a); break;
            case kVarPairedStagedR96: (g5 ? k_hop_x2s_r96<1> : k_hop_x2s_r96<0>)<<<grid, c.block, sm, s>>>(a); break;
            case kVarPairedR96: (g5 ? k_hop_x2_r96<1> : k_hop_x2_r96<0>)<<<grid, c.block, 0, s>>>(a); break;
            default: (g5 ? k_hop_x2<1> : k_hop_x2<0>)<<<grid, c.block, 0, s>>>(a); break;
            }
            st = check_launch(ctx, "paired hop kernel");
            return true;
        } else if constexpr (PREC == kF64) {
            // adjoint (quaternion or stored 3x3 links): (re, im) lanes
            if (c.variant != kVarPaired && c.variant != kVarPairedStaged && c.variant != kVarPairedR96) return false;
            const bool g5 = a.g5_in != 0;
            if (c.variant == kVarPairedR96) {
                // for the adjoint: the form with 168 registers
                (g5 ? k_hop_x2a_big<REP, 1> : k_hop_x2a_big<REP, 0>)<<<grid, c.block, 0, s>>>(a);
                st = check_launch(ctx, "paired adjoint hop kernel (168 registers)");
                return true;
            }
            if constexpr (REP == kRepAdj) {
                if (c.variant == kVarPairedStaged) {
                    using S = Stage<kRepAdj, kF64>;
                    static bool attr_set = false;
                    if (!attr_set) {
                        for (auto f : {k_hop_x2as<0>, k_hop_x2as<1>})
                            cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)S::smem_bytes(256));
                        attr_set = true;
                    }
                    (g5 ? k_hop_x2as<1> : k_hop_x2as<0>)<<<grid, c.block, S::smem_bytes(c.block), s>>>(a);
                    st = check_launch(ctx, "paired adjoint hop kernel");
                    return true;
                }
            }
            (g5 ? k_hop_x2a<REP, 1> : k_hop_x2a<REP, 0>)<<<grid, c.block, 0, s>>>(a);
            st = check_launch(ctx, "paired adjoint hop kernel");
            return true;
        } else if constexpr (REP == kRepFund) {
            // FP32 arithmetic: the register-capped forms are not built (the
            // kernels need far fewer registers): those variants run the plain kernel
            if (c.variant != kVarPaired && c.variant != kVarPairedStaged) return false;
            using S = Stage<kRepFund, PREC>;
            static bool attr_set = false;
            if (!attr_set) {
                for (auto f : {k_hop_f2s<PREC, 0>, k_hop_f2s<PREC, 1>})
                    cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::smem_bytes(256));
                attr_set = true;
            }
            const bool g5 = a.g5_in != 0;
            if (c.variant == kVarPairedStaged)
                (g5 ? k_hop_f2s<PREC, 1> : k_hop_f2s<PREC, 0>)<<<grid, c.block, S::smem_bytes(c.block), s>>>(a);
            else
                (g5 ? k_hop_f2<PREC, 1> : k_hop_f2<PREC, 0>)<<<grid, c.block, 0, s>>>(a);
            st = check_launch(ctx, "paired hop kernel");
            return true;
        }
        return false;
    }
};

} // namespace

namespace hr {

void launch_hop_clover_paired(hr_ctx *ctx, const HopArgs &a, int grid, int block, cudaStream_t s, hr_status &st)
{
    using S = Stage<kRepFund, kF64>;
    static bool attr_set = false;
    if (!attr_set) {
        for (auto f : {k_hop_x2s_clov<0>, k_hop_x2s_clov<1>})
            cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::smem_bytes(256));
        attr_set = true;
    }
    (a.g5_in ? k_hop_x2s_clov<1> : k_hop_x2s_clov<0>)<<<grid, block, S::smem_bytes(block), s>>>(a);
    st = check_launch(ctx, "paired hop kernel (clover epilogue)");
}

bool launch_hop_paired(hr_ctx *ctx, const Geom &g, int rep, int prec, const HopArgs &a, HopChoice c, int grid,
                       cudaStream_t s, hr_status &st)
{
    return for_config<Launch>(rep, prec, ctx, g, a, c, grid, s, st);
}

} // namespace hr
