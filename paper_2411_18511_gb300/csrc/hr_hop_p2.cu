// hr_hop_p2.cu -- the FP32-arithmetic fundamental hop with two output sites per
// thread in the lanes of the packed f32x2 FMA (variants 16 and 17; FP32 and
// binary16 storage).
//
// The FP32 and FP16 hops move 256 and 136 bytes per output site (the
// multi-RHS FP32 hop 132 per virtual site at 32 right-hand sides), and at
// those byte counts the instruction issue, not HBM, sets their pace: a
// thread per site spends 48 scalar FMAs per direction on the colour product
// and the rebuild.  Here a thread takes the virtual sites j and j + 32 (the
// same lane of two consecutive 32-site blocks, so every load instruction of a
// warp still reads contiguous 512-byte runs) and computes both at once: each
// packed FMA does one operation of each site.  The projection runs per site
// (binary16: in half2 on the stored words, as in variants 14 / 15; FP32:
// scalar adds) and its results are written straight into the two lanes; the
// links of the two sites form the coefficient pairs; the neighbour scale of
// the binary16 layout rides on the accumulating FMAs.  Arithmetic is that of
// the one-site kernels (agreement to rounding).  When the site count is not a
// multiple of 64 the second lane of the last pairs repeats the first site and
// is not stored.
//
// Variant 16: registers as the compiler likes; 17: capped at 96.
#include "hr_hop_fam.h"
#include "hr_hop_x2.cuh"

using namespace hr;

namespace {

__device__ __forceinline__ float2 pr(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2f(float2 a, float2 b, float2 zero) { return __ffma2_rn(a, b, zero); }

// h (re, im) of one site for spins t = 0, 1 and colours c = 0, 1
struct Half {
    float re[2][2], im[2][2]; // [t][c]
};

// h_t = s_t + i^C s_pi from the FP32 layout: spin s is the float4 (c0.re, c1.re, c0.im, c1.im)
template <int C>
__device__ __forceinline__ void f32_project(const float4 &s, const float4 &y, float (&re)[2], float (&im)[2])
{
    if constexpr (C == 0) {
        re[0] = s.x + y.x; re[1] = s.y + y.y; im[0] = s.z + y.z; im[1] = s.w + y.w;
    } else if constexpr (C == 1) {
        re[0] = s.x - y.z; re[1] = s.y - y.w; im[0] = s.z + y.x; im[1] = s.w + y.y;
    } else if constexpr (C == 2) {
        re[0] = s.x - y.x; re[1] = s.y - y.y; im[0] = s.z - y.z; im[1] = s.w - y.w;
    } else {
        re[0] = s.x + y.z; re[1] = s.y + y.w; im[0] = s.z - y.x; im[1] = s.w - y.y;
    }
}

// one site's projected half spinor, its link and its scale for direction (MU, FWD)
template <int MU, bool FWD, bool NEG, int PREC>
__device__ __forceinline__ void p2_site(const HopArgs &a, const float *nrm, int site_link, int link_par, int jn,
                                        Half &h, float (&q)[4], float &sc)
{
    using D = X2Dir<MU, FWD>;
    constexpr int F = NEG ? 2 : 0;
    if constexpr (PREC == kF16) {
        const uint4 *sp = (const uint4 *)a.in;
        const uint4 w0 = __ldg(sp + vec_index(jn, 0, 2));
        const uint4 w1 = __ldg(sp + vec_index(jn, 1, 2));
        sc = __ldg(nrm + jn);
        const uint32_t u[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
        __half2 h0re, h0im, h1re, h1im;
        h2_project<(D::c0 + F) & 3>(as_h2(u[0]), as_h2(u[1]), as_h2(u[2 * D::pi0]), as_h2(u[2 * D::pi0 + 1]), h0re,
                                    h0im);
        h2_project<(D::c1 + F) & 3>(as_h2(u[2]), as_h2(u[3]), as_h2(u[2 * D::pi1]), as_h2(u[2 * D::pi1 + 1]), h1re,
                                    h1im);
        const float2 r0 = __half22float2(h0re), i0 = __half22float2(h0im);
        const float2 r1 = __half22float2(h1re), i1 = __half22float2(h1im);
        h.re[0][0] = r0.x; h.re[0][1] = r0.y; h.im[0][0] = i0.x; h.im[0][1] = i0.y;
        h.re[1][0] = r1.x; h.re[1][1] = r1.y; h.im[1][0] = i1.x; h.im[1][1] = i1.y;
    } else {
        const float4 *sp = (const float4 *)a.in;
        float4 s[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) s[v] = __ldg(sp + vec_index(jn, v, 4));
        sc = 1.f;
        f32_project<(D::c0 + F) & 3>(s[0], s[D::pi0], h.re[0], h.im[0]);
        f32_project<(D::c1 + F) & 3>(s[1], s[D::pi1], h.re[1], h.im[1]);
    }
    load_quat<PREC>(a.gauge, a.g.nblk_g, link_par, MU, site_link, q);
}

// acc (+)= i^C (sc r) on lane pairs; SC = (sc1, sc2), NS = -SC
template <int C, bool FIRST>
__device__ __forceinline__ void p2_acc(float2 &are, float2 &aim, float2 rre, float2 rim, float2 SC, float2 NS,
                                       float2 Z)
{
    if constexpr (FIRST) {
        if constexpr (C == 0) { are = mul2f(rre, SC, Z); aim = mul2f(rim, SC, Z); }
        else if constexpr (C == 1) { are = mul2f(rim, NS, Z); aim = mul2f(rre, SC, Z); }
        else if constexpr (C == 2) { are = mul2f(rre, NS, Z); aim = mul2f(rim, NS, Z); }
        else { are = mul2f(rim, SC, Z); aim = mul2f(rre, NS, Z); }
    } else {
        if constexpr (C == 0) { are = fma2(rre, SC, are); aim = fma2(rim, SC, aim); }
        else if constexpr (C == 1) { are = fma2(rim, NS, are); aim = fma2(rre, SC, aim); }
        else if constexpr (C == 2) { are = fma2(rre, NS, are); aim = fma2(rim, NS, aim); }
        else { are = fma2(rim, SC, are); aim = fma2(rre, NS, aim); }
    }
}

// both sites' term of direction (MU, FWD): acc[spin][colour] (re, im) lane pairs
template <int MU, bool FWD, bool FIRST, bool NEG, int PREC>
__device__ __forceinline__ void p2_term(const HopArgs &a, const K2 &k, const float *nrm, int sl1, int sl2,
                                        int link_par, int jn1, int jn2, float2 (&are)[4][2], float2 (&aim)[4][2])
{
    using D = X2Dir<MU, FWD>;
    constexpr int F = NEG ? 2 : 0;
    Half h1, h2;
    float q1[4], q2[4], sc1, sc2;
    p2_site<MU, FWD, NEG, PREC>(a, nrm, sl1, link_par, jn1, h1, q1, sc1);
    p2_site<MU, FWD, NEG, PREC>(a, nrm, sl2, link_par, jn2, h2, q2, sc2);
    // coefficient pairs; U (FWD) or U^+: the signs of a1, a2, a3 flip
    const float2 A0 = pr(q1[0], q2[0]);
    const float2 P1 = FWD ? pr(q1[1], q2[1]) : pr(-q1[1], -q2[1]), M1 = FWD ? pr(-q1[1], -q2[1]) : pr(q1[1], q2[1]);
    const float2 P2 = FWD ? pr(q1[2], q2[2]) : pr(-q1[2], -q2[2]), M2 = FWD ? pr(-q1[2], -q2[2]) : pr(q1[2], q2[2]);
    const float2 P3 = FWD ? pr(q1[3], q2[3]) : pr(-q1[3], -q2[3]), M3 = FWD ? pr(-q1[3], -q2[3]) : pr(q1[3], q2[3]);
    const float2 SC = pr(sc1, sc2), NS = pr(-sc1, -sc2);
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const float2 h0r = pr(h1.re[t][0], h2.re[t][0]), h0i = pr(h1.im[t][0], h2.im[t][0]);
        const float2 h1r = pr(h1.re[t][1], h2.re[t][1]), h1i = pr(h1.im[t][1], h2.im[t][1]);
        // r = U h (su2_mul): c0 = a0 h0 + i a3 h0 + (a2 + i a1) h1, c1 = (-a2 + i a1) h0 + a0 h1 - i a3 h1
        float2 r0r = mul2f(A0, h0r, k.zero);
        r0r = fma2(M3, h0i, r0r);
        r0r = fma2(P2, h1r, r0r);
        r0r = fma2(M1, h1i, r0r);
        float2 r0i = mul2f(A0, h0i, k.zero);
        r0i = fma2(P3, h0r, r0i);
        r0i = fma2(P2, h1i, r0i);
        r0i = fma2(P1, h1r, r0i);
        float2 r1r = mul2f(A0, h1r, k.zero);
        r1r = fma2(P3, h1i, r1r);
        r1r = fma2(M2, h0r, r1r);
        r1r = fma2(M1, h0i, r1r);
        float2 r1i = mul2f(A0, h1i, k.zero);
        r1i = fma2(M3, h1r, r1i);
        r1i = fma2(M2, h0i, r1i);
        r1i = fma2(P1, h0r, r1i);
        // upper spin t, and the lower spin(s) rebuilt from r_t
        p2_acc<F, FIRST>(are[t][0], aim[t][0], r0r, r0i, SC, NS, k.zero);
        p2_acc<F, FIRST>(are[t][1], aim[t][1], r1r, r1i, SC, NS, k.zero);
        if (D::rho0 == t) {
            p2_acc<(D::d0 + F) & 3, FIRST>(are[2][0], aim[2][0], r0r, r0i, SC, NS, k.zero);
            p2_acc<(D::d0 + F) & 3, FIRST>(are[2][1], aim[2][1], r1r, r1i, SC, NS, k.zero);
        }
        if (D::rho1 == t) {
            p2_acc<(D::d1 + F) & 3, FIRST>(are[3][0], aim[3][0], r0r, r0i, SC, NS, k.zero);
            p2_acc<(D::d1 + F) & 3, FIRST>(are[3][1], aim[3][1], r1r, r1i, SC, NS, k.zero);
        }
    }
}

template <int MU, bool FIRST, bool NEG, int PREC>
__device__ __forceinline__ void p2_dir(const HopArgs &a, const K2 &k, const float *nrm, int i1, int i2, int rr,
                                       const SiteNb &n1, const SiteNb &n2, float2 (&are)[4][2], float2 (&aim)[4][2])
{
    const int l = a.g.lrhs;
    p2_term<MU, true, FIRST, NEG, PREC>(a, k, nrm, i1, i2, a.p, (n1.fwd[MU] << l) + rr, (n2.fwd[MU] << l) + rr, are,
                                        aim);
    p2_term<MU, false, false, NEG, PREC>(a, k, nrm, n1.bwd[MU], n2.bwd[MU], 1 - a.p, (n1.bwd[MU] << l) + rr,
                                         (n2.bwd[MU] << l) + rr, are, aim);
}

template <int PREC, int G5IN>
__device__ __forceinline__ void p2_body(const HopArgs &a)
{
    constexpr bool NEG = G5IN != 0;
    if ((a.gate && *a.gate == 0.0) || (a.done && *a.done != 0.0)) return;
    const K2 k = make_k2(a.unit, a.nil);
    const Geom &g = a.g;
    const int nv = g.vh << g.lrhs;
    const int npairs = ((nv + 63) >> 6) << 5; // 32 pairs per 64 virtual sites
    const int stride = gridDim.x * blockDim.x;
    const float *nrm =
        PREC == kF16 ? (const float *)((const char *)a.in + SpinorLayout<2, kF16>::data_bytes(g.nblk_s)) : nullptr;
    const float be = a.beta.h;
    const float bu = a.g5_out ? -be : be;
    const float al = a.alpha.h;
    SqAcc<float> red;
    for (int P = blockIdx.x * blockDim.x + threadIdx.x; P < npairs; P += stride) {
        const int j1 = ((P >> 5) << 6) + (P & 31);
        if (j1 >= nv) continue;
        const bool two = j1 + 32 < nv;
        const int j2 = two ? j1 + 32 : j1; // the last pairs may repeat the first site
        const int rr = j1 & (g.nrhs - 1);  // = j2's: 32 is a multiple of the RHS count
        const int i1 = j1 >> g.lrhs, i2 = j2 >> g.lrhs;
        SiteNb n1, n2;
        site_neighbours(g, i1, a.p, n1);
        site_neighbours(g, i2, a.p, n2);
        float2 are[4][2], aim[4][2];
        p2_dir<0, true, NEG, PREC>(a, k, nrm, i1, i2, rr, n1, n2, are, aim);
        p2_dir<1, false, NEG, PREC>(a, k, nrm, i1, i2, rr, n1, n2, are, aim);
        p2_dir<2, false, NEG, PREC>(a, k, nrm, i1, i2, rr, n1, n2, are, aim);
        p2_dir<3, false, NEG, PREC>(a, k, nrm, i1, i2, rr, n1, n2, are, aim);
        cpx<float> o1[4][2], o2[4][2];
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                o1[t][c] = {are[t][c].x, aim[t][c].x};
                o2[t][c] = {are[t][c].y, aim[t][c].y};
            }
        hop_epilogue<PREC>(a, j1, o1, al, be, bu, red);
        if (two) hop_epilogue<PREC>(a, j2, o2, al, be, bu, red);
    }
    if (a.fin) {
        __shared__ double smem[32 * 32];
        __shared__ double sums[32];
        if (grid_reduce(red, g.nrhs, a.red, sums, smem)) finish_reduction(a.fin, sums, g.nrhs, a.scal);
    }
}

template <int PREC, int G5IN> __global__ void __launch_bounds__(256) k_hop_p2(HopArgs a) { p2_body<PREC, G5IN>(a); }
template <int PREC, int G5IN> __global__ void __maxnreg__(96) k_hop_p2_r96(HopArgs a) { p2_body<PREC, G5IN>(a); }

template <int PREC>
void launch_p2(const HopArgs &a, HopChoice c, int grid, cudaStream_t s)
{
    const bool g5 = a.g5_in != 0;
    if (c.variant == kVarPairSitesR96) (g5 ? k_hop_p2_r96<PREC, 1> : k_hop_p2_r96<PREC, 0>)<<<grid, c.block, 0, s>>>(a);
    else (g5 ? k_hop_p2<PREC, 1> : k_hop_p2<PREC, 0>)<<<grid, c.block, 0, s>>>(a);
}

} // namespace

namespace hr {

bool launch_hop_pair_sites(hr_ctx *ctx, const Geom &g, int rep, int prec, const HopArgs &a, HopChoice c, int,
                           cudaStream_t s, hr_status &st)
{
    if (rep != HR_FUND || (prec != kF32 && prec != kF16)) return false;
    // one thread per pair of virtual sites
    const long long nv = (long long)g.vh << g.lrhs;
    const long long npairs = ((nv + 63) >> 6) << 5;
    const int grid = grid_for(npairs, c.block, a.fin ? kMaxBlocks : (1 << 30));
    if (prec == kF32) launch_p2<kF32>(a, c, grid, s);
    else launch_p2<kF16>(a, c, grid, s);
    st = check_launch(ctx, "two-site hop kernel");
    return true;
}

} // namespace hr
