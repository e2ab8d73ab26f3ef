// hr_internal.cuh -- shared device code of libhirep_gb300: lattice geometry,
// packed field layouts, complex arithmetic and the spin/colour algebra of the
// Wilson hopping term.
//
// Operator (arXiv:2411.18511 names the unimproved Wilson-Dirac operator in
// Sec. 2.1 / Table 1 without writing it; this is the textbook form):
//   (H psi)(x) = sum_mu (1-g_mu) U_mu(x) psi(x+mu) + (1+g_mu) U_mu(x-mu)^+ psi(x-mu)
// in the chiral basis g_0 = [[0,1],[1,0]], g_k = [[0,-i s_k],[i s_k,0]].
//
// Packed layouts (device, opaque to callers)
// ------------------------------------------
// Sites of one parity are numbered by their even-odd index i = lex/2, where
// lex = ((x0*L1 + x1)*L2 + x2)*L3 + x3; a multi-RHS field numbers "virtual
// sites" j = i*N + r (r = right-hand side, N a power of two <= 32).  Fields are
// array-of-structure-of-arrays in blocks of 32 virtual sites: one 16-byte
// vector v of site j sits at vector index ((j/32)*NVEC + v)*32 + j%32, so a
// warp reading one vector of 32 consecutive sites reads 512 contiguous bytes.
//   spinor FP64: NVEC = 4*NC float4, 8 bytes per real like binary64, in
//                double-float parts.  NC = 2 (colour-paired): spin s has vector
//                2s = hi parts (c0.re, c1.re, c0.im, c1.im), vector 2s+1 = the
//                lo parts in the same order, so a vector holds the two colours
//                of one part side by side (what the packed f32x2 hop uses).
//                NC = 3: one complex per float4, (re.h, im.h, re.l, im.l).
//   spinor FP32: NVEC = 2*NC float4, FP16: NVEC = NC uint4 (binary16, followed
//                by one float scale per site, the site's max |component|): the
//                8*NC reals in packed order -- NC = 2 (colour-paired): spin s
//                gives (c0.re, c1.re, c0.im, c1.im); NC = 3: (re, im) of each
//                (spin, colour) in turn.
//   gauge (quaternion links): link (p, mu, i) in slot L = (p*4+mu)*nblk + i/32,
//     FP64 two float4 (the four hi parts, then the four lo parts) at
//     (L*2+v)*32 + i%32, FP32 one float4, FP16 one uint2
//   gauge HR_ADJ_MAT: 9 reals R_ab at (L*9 + 3a+b)*32 + i%32 (FP64: float2 h, l)
// where nblk = ceil(V_h/32) for the gauge and ceil(V_h*N/32) for spinors.
#pragma once

#include <cmath>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "hirep_gb300.h"

namespace hr {

constexpr int kRepFund = 0, kRepAdj = 1, kRepAdjMat = 2;
constexpr int kF64 = 0, kF32 = 1, kF16 = 2;

template <int REP> struct RepTraits { static constexpr int NC = (REP == kRepFund) ? 2 : 3; };

// ---------------------------------------------------------------- geometry

// Division by a launch-invariant divisor d as a multiply and a shift:
// q = (n * m) >> s with m = ceil(2^(31+l) / d), 2^l >= d, exact for 0 <= n < 2^31
// (the rounding error n (m d - 2^(31+l)) / 2^(31+l) d stays below 1/d).
struct FastDiv {
    unsigned m;
    int s;
};
inline FastDiv make_fastdiv(unsigned d)
{
    int l = 0;
    while ((1u << l) < d) ++l;
    unsigned long long m = ((1ULL << (31 + l)) + d - 1) / d;
    FastDiv f;
    f.m = (unsigned)m;
    f.s = 31 + l;
    return f;
}
__device__ __forceinline__ int fdiv(int n, FastDiv f) { return (int)(((unsigned long long)(unsigned)n * f.m) >> f.s); }

// A double-precision scalar split on the host into two floats, so kernels get
// launch constants in any of their arithmetic types without FP64 conversions.
struct coef2 {
    float h, l;
};
inline coef2 make_coef(double x)
{
    coef2 c;
    c.h = (float)x;
    c.l = (float)(x - (double)c.h);
    return c;
}

struct Geom {
    int d[4];   // T, L1, L2, L3
    int h3;     // L3 / 2
    int vh;     // sites per parity
    int nrhs;   // right-hand sides (power of two)
    int lrhs;   // log2(nrhs)
    int nblk_g; // 32-site blocks of the gauge (per parity and direction)
    int nblk_s; // 32-virtual-site blocks of a spinor field of one parity
    int bc;     // antiperiodic directions (bit mu); used where links are packed
    FastDiv div_h3, div_d2, div_d1;
    // twisted boundaries: e^{i theta_mu} = tw_c + i tw_s (each a float pair,
    // h + l), applied by the twisted hop kernel only; twisted = 0 when all
    // four angles are zero
    int twisted;
    coef2 tw_c[4], tw_s[4];
};

inline Geom make_geom(const hr_lattice &lat, int nrhs)
{
    Geom g;
    for (int k = 0; k < 4; ++k) g.d[k] = lat.dims[k];
    g.h3 = lat.dims[3] / 2;
    long long v = (long long)lat.dims[0] * lat.dims[1] * lat.dims[2] * lat.dims[3];
    g.vh = (int)(v / 2);
    g.nrhs = nrhs;
    int l = 0;
    while ((1 << l) < nrhs) ++l;
    g.lrhs = l;
    g.nblk_g = (g.vh + 31) / 32;
    g.nblk_s = (int)(((long long)g.vh * nrhs + 31) / 32);
    g.bc = lat.bc;
    g.div_h3 = make_fastdiv((unsigned)(g.h3 > 0 ? g.h3 : 1));
    g.div_d2 = make_fastdiv((unsigned)(g.d[2] > 0 ? g.d[2] : 1));
    g.div_d1 = make_fastdiv((unsigned)(g.d[1] > 0 ? g.d[1] : 1));
    g.twisted = 0;
    for (int k = 0; k < 4; ++k) {
        g.twisted |= lat.theta[k] != 0.0;
        g.tw_c[k] = make_coef(std::cos(lat.theta[k]));
        g.tw_s[k] = make_coef(std::sin(lat.theta[k]));
    }
    return g;
}

// Coordinates and neighbours of the site with even-odd index i and parity p.
struct SiteNb {
    int fwd[4]; // even-odd index of x + mu (other parity)
    int bwd[4]; // even-odd index of x - mu (other parity)
};

__device__ __forceinline__ void site_neighbours(const Geom &g, int i, int p, SiteNb &nb)
{
    const int h3 = g.h3;
    int row = fdiv(i, g.div_h3);
    int k = i - row * h3;
    int r1 = fdiv(row, g.div_d2);
    int x2 = row - r1 * g.d[2];
    int x0 = fdiv(r1, g.div_d1);
    int x1 = r1 - x0 * g.d[1];
    int odd3 = (x0 + x1 + x2 + p) & 1; // x3 = 2k + odd3
    // direction 3 (fastest): stays in the row, wraps within it
    int base = row * h3;
    nb.fwd[3] = odd3 ? (k + 1 == h3 ? base : i + 1) : i;
    nb.bwd[3] = odd3 ? i : (k == 0 ? base + h3 - 1 : i - 1);
    // directions 2, 1, 0: move whole rows
    const int s2 = h3, s1 = g.d[2] * h3, s0 = g.d[1] * g.d[2] * h3;
    nb.fwd[2] = (x2 + 1 == g.d[2]) ? i - (g.d[2] - 1) * s2 : i + s2;
    nb.bwd[2] = (x2 == 0) ? i + (g.d[2] - 1) * s2 : i - s2;
    nb.fwd[1] = (x1 + 1 == g.d[1]) ? i - (g.d[1] - 1) * s1 : i + s1;
    nb.bwd[1] = (x1 == 0) ? i + (g.d[1] - 1) * s1 : i - s1;
    nb.fwd[0] = (x0 + 1 == g.d[0]) ? i - (g.d[0] - 1) * s0 : i + s0;
    nb.bwd[0] = (x0 == 0) ? i + (g.d[0] - 1) * s0 : i - s0;
}

// lexicographic index of the site with even-odd index i and parity p
__device__ __forceinline__ long long eo_to_lex(const Geom &g, int i, int p)
{
    int row = fdiv(i, g.div_h3);
    int k = i - row * g.h3;
    int r1 = fdiv(row, g.div_d2);
    int x2 = row - r1 * g.d[2];
    int x0 = fdiv(r1, g.div_d1);
    int x1 = r1 - x0 * g.d[1];
    int odd3 = (x0 + x1 + x2 + p) & 1;
    return (long long)row * g.d[3] + 2 * k + odd3;
}

// ---------------------------------------------------------------- complex

template <class T> struct cpx {
    T re, im;
};

template <class T> __device__ __forceinline__ cpx<T> cadd(cpx<T> a, cpx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <class T> __device__ __forceinline__ cpx<T> csub(cpx<T> a, cpx<T> b) { return {a.re - b.re, a.im - b.im}; }
// a + i b, a - i b
template <class T> __device__ __forceinline__ cpx<T> cadd_i(cpx<T> a, cpx<T> b) { return {a.re - b.im, a.im + b.re}; }
template <class T> __device__ __forceinline__ cpx<T> csub_i(cpx<T> a, cpx<T> b) { return {a.re + b.im, a.im - b.re}; }

// ---------------------------------------------------------------- double-float
// FP64-accuracy arithmetic on the FP32 pipes (GB300 executes FP64 FMA at about
// 1/60 of the FP32 rate).  A value is the unevaluated sum h + l of two floats
// (Dekker 1971); sums use Knuth's TwoSum, products the FMA-based TwoProduct.
// Results are kept unnormalised inside a kernel (|l| stays of the order of
// 2^-24 times the operands) and renormalised with TwoSum before they are
// stored, which keeps a relative accuracy of about 2^-47 per operation.

struct dd {
    float h, l;
    dd() = default;
    __host__ __device__ constexpr dd(float h_, float l_) : h(h_), l(l_) {}
    __host__ __device__ constexpr dd(float x) : h(x), l(0.f) {}
};

__device__ __forceinline__ dd two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float v = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
    return dd(s, e);
}
__device__ __forceinline__ dd dd_norm(dd a) { return two_sum(a.h, a.l); }
__device__ __forceinline__ dd operator+(dd a, dd b)
{
    dd s = two_sum(a.h, b.h);
    s.l = __fadd_rn(s.l, __fadd_rn(a.l, b.l));
    return s;
}
__device__ __forceinline__ dd operator-(dd a) { return dd(-a.h, -a.l); }
__device__ __forceinline__ dd operator-(dd a, dd b) { return a + (-b); }
__device__ __forceinline__ dd operator*(dd a, dd b)
{
    float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return dd(p, e);
}
__device__ __forceinline__ dd operator*(float a, dd b)
{
    float p = __fmul_rn(a, b.h);
    float e = __fmaf_rn(a, b.h, -p);
    e = __fmaf_rn(a, b.l, e);
    return dd(p, e);
}
__device__ __forceinline__ dd &operator+=(dd &a, dd b) { return a = a + b; }
__device__ __forceinline__ dd &operator-=(dd &a, dd b) { return a = a - b; }
// conversions through the FP64 unit: only outside hot loops
__device__ __forceinline__ dd dd_from_double(double x)
{
    float h = __double2float_rn(x);
    return dd(h, __double2float_rn(x - (double)h));
}
__device__ __forceinline__ double dd_to_double(dd a) { return (double)a.h + (double)a.l; }

template <class T> struct Real;
template <> struct Real<float> {
    __device__ static float from_coef(coef2 c) { return c.h; }
    __device__ static float from_double(double x) { return (float)x; }
    __device__ static float from_float(float x) { return x; }
    __device__ static double to_double(float x) { return (double)x; }
    __device__ static float to_float(float x) { return x; }
    __device__ static dd to_dd(float x) { return dd(x); }
};
template <> struct Real<double> {
    __device__ static double from_coef(coef2 c) { return (double)c.h + (double)c.l; }
    __device__ static double from_double(double x) { return x; }
    __device__ static double from_float(float x) { return (double)x; }
    __device__ static double to_double(double x) { return x; }
    __device__ static float to_float(double x) { return (float)x; }
    __device__ static dd to_dd(double x) { return dd_from_double(x); }
};
template <> struct Real<dd> {
    __device__ static dd from_coef(coef2 c) { return dd(c.h, c.l); }
    __device__ static dd from_double(double x) { return dd_from_double(x); }
    __device__ static dd from_float(float x) { return dd(x); }
    __device__ static double to_double(dd x) { return dd_to_double(x); }
    __device__ static float to_float(dd x) { return __fadd_rn(x.h, x.l); }
    __device__ static dd to_dd(dd x) { return dd_norm(x); }
};

// Accumulator of sums of squares with the precision of T, finished in double.
template <class T> struct SqAcc;
template <> struct SqAcc<float> {
    float s = 0.f;
    __device__ void add(float x) { s = __fmaf_rn(x, x, s); }
    __device__ double get() const { return (double)s; }
};
template <> struct SqAcc<double> {
    double s = 0.0;
    __device__ void add(double x) { s += x * x; }
    __device__ double get() const { return s; }
};
template <> struct SqAcc<dd> {
    dd s = dd(0.f);
    __device__ void add(dd x)
    {
        // renormalise first: after cancellation (a residual near convergence)
        // |l| may exceed |h|, and h^2 + 2hl without l^2 could then be negative
        x = dd_norm(x);
        float p = __fmul_rn(x.h, x.h);
        float e = __fmaf_rn(x.h, x.h, -p);
        e = __fmaf_rn(__fadd_rn(x.h, x.h), x.l, e);
        s += dd(p, e);
    }
    __device__ double get() const { return dd_to_double(s); }
};

// ---------------------------------------------------------------- value range
// The FP64 layouts hold each real as a pair of floats, so they keep the float
// exponent range: a value v keeps its 48 significant bits while its low part
// is a normal float (|v| >= 2^-102), and an operator's sums stay finite while
// the inputs stay well below the float maximum 2^128.  The pack kernels accept
// canonical values up to 2^120 in magnitude (room for the growth of a few
// operator applications) and flag larger or non-finite ones in the context's
// pack status word; the solvers rescale their source by a power of two, which
// is exact, so that the vectors they iterate are of order one.
constexpr unsigned kPackAboveRange = 2u, kPackNonFinite = 4u;
__device__ __forceinline__ unsigned pack_range_flags(double v)
{
    if (!isfinite(v)) return kPackNonFinite;
    return fabs(v) > 0x1p120 ? kPackAboveRange : 0u;
}

// ---------------------------------------------------------------- layouts

template <int PREC> struct PrecTraits;
// FP64 fields are stored as double-float pairs: 8 bytes per real, like binary64
template <> struct PrecTraits<kF64> { using T = dd; static constexpr int W = 2; };
template <> struct PrecTraits<kF32> { using T = float; static constexpr int W = 4; };
template <> struct PrecTraits<kF16> { using T = float; static constexpr int W = 8; };

template <int NC, int PREC> struct SpinorLayout {
    static constexpr int NR = 8 * NC;                    // reals per site
    static constexpr int NVEC = NR / PrecTraits<PREC>::W; // 16-byte vectors per site
    __host__ __device__ static size_t data_bytes(int nblk) { return (size_t)nblk * 32 * NVEC * 16; }
    static size_t bytes(int nblk)
    {
        size_t b = data_bytes(nblk);
        if (PREC == kF16) b += (size_t)nblk * 32 * sizeof(float);
        return (b + 255) & ~(size_t)255;
    }
};

__device__ __forceinline__ size_t vec_index(int j, int v, int nvec)
{
    return ((size_t)(j >> 5) * nvec + v) * 32 + (j & 31);
}

// position of Re / Im of (spin sp, colour c) among the 8 NC reals of a site in
// the packed order of the FP32 / FP16 layouts (and of the FP64 hi/lo vectors
// when NC = 2)
template <int NC> __host__ __device__ constexpr int packed_re(int sp, int c)
{
    return NC == 2 ? 4 * sp + c : 2 * (NC * sp + c);
}
template <int NC> __host__ __device__ constexpr int packed_im(int sp, int c)
{
    return NC == 2 ? 4 * sp + 2 + c : 2 * (NC * sp + c) + 1;
}
template <int NC, class T>
__device__ __forceinline__ void values_from_packed(const float *r, float sc, cpx<T> (&s)[4][NC])
{
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int c = 0; c < NC; ++c)
            s[sp][c] = {Real<T>::from_float(r[packed_re<NC>(sp, c)] * sc),
                        Real<T>::from_float(r[packed_im<NC>(sp, c)] * sc)};
}
template <int NC, class T> __device__ __forceinline__ void values_to_packed(const cpx<T> (&s)[4][NC], float *r)
{
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            r[packed_re<NC>(sp, c)] = Real<T>::to_float(s[sp][c].re);
            r[packed_im<NC>(sp, c)] = Real<T>::to_float(s[sp][c].im);
        }
}
__device__ __forceinline__ void float4_to_floats(const float4 &w, float *f)
{
    f[0] = w.x;
    f[1] = w.y;
    f[2] = w.z;
    f[3] = w.w;
}
// the 8 binary16 reals of one uint4, in order
__device__ __forceinline__ void halves_to_floats(const uint4 &w, float *f)
{
    const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float2 t = __half22float2(*reinterpret_cast<const __half2 *>(&u[q]));
        f[2 * q] = t.x;
        f[2 * q + 1] = t.y;
    }
}

// FP64 vectors <-> values (layout above)
template <int NC, class T>
__device__ __forceinline__ void f64_from_vecs(const float4 *w, cpx<T> (&s)[4][NC])
{
    auto val = [](float h, float l) -> T {
        if constexpr (std::is_same<T, dd>::value) return dd(h, l);
        else return Real<T>::from_double(dd_to_double(dd(h, l)));
    };
    if constexpr (NC == 2) {
#pragma unroll
        for (int sp = 0; sp < 4; ++sp) {
            const float4 hi = w[2 * sp], lo = w[2 * sp + 1];
            s[sp][0] = {val(hi.x, lo.x), val(hi.z, lo.z)};
            s[sp][1] = {val(hi.y, lo.y), val(hi.w, lo.w)};
        }
    } else {
        cpx<T> *flat = &s[0][0];
#pragma unroll
        for (int v = 0; v < 4 * NC; ++v) flat[v] = {val(w[v].x, w[v].z), val(w[v].y, w[v].w)};
    }
}
template <int NC, class T>
__device__ __forceinline__ void f64_to_vecs(const cpx<T> (&s)[4][NC], float4 *w)
{
    if constexpr (NC == 2) {
#pragma unroll
        for (int sp = 0; sp < 4; ++sp) {
            const dd r0 = Real<T>::to_dd(s[sp][0].re), i0 = Real<T>::to_dd(s[sp][0].im);
            const dd r1 = Real<T>::to_dd(s[sp][1].re), i1 = Real<T>::to_dd(s[sp][1].im);
            w[2 * sp] = make_float4(r0.h, r1.h, i0.h, i1.h);
            w[2 * sp + 1] = make_float4(r0.l, r1.l, i0.l, i1.l);
        }
    } else {
        const cpx<T> *flat = &s[0][0];
#pragma unroll
        for (int v = 0; v < 4 * NC; ++v) {
            const dd re = Real<T>::to_dd(flat[v].re), im = Real<T>::to_dd(flat[v].im);
            w[v] = make_float4(re.h, im.h, re.l, im.l);
        }
    }
}

template <int NC, int PREC, class T>
__device__ __forceinline__ void load_spinor(const void *base, int nblk, int j, cpx<T> (&s)[4][NC])
{
    using L = SpinorLayout<NC, PREC>;
    constexpr int NV = L::NVEC;
    if constexpr (PREC == kF64) {
        const float4 *p = (const float4 *)base;
        float4 w[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) w[v] = __ldg(p + vec_index(j, v, NV));
        f64_from_vecs<NC>(w, s);
    } else if constexpr (PREC == kF32) {
        const float4 *p = (const float4 *)base;
        float r[8 * NC];
#pragma unroll
        for (int v = 0; v < NV; ++v) float4_to_floats(__ldg(p + vec_index(j, v, NV)), &r[4 * v]);
        values_from_packed<NC>(r, 1.f, s);
    } else {
        const uint4 *p = (const uint4 *)base;
        const float *nrm = (const float *)((const char *)base + L::data_bytes(nblk));
        const float sc = __ldg(nrm + j);
        float r[8 * NC];
#pragma unroll
        for (int v = 0; v < NV; ++v) halves_to_floats(__ldg(p + vec_index(j, v, NV)), &r[8 * v]);
        values_from_packed<NC>(r, sc, s);
    }
}

// As load_spinor, but a binary16 site is returned unscaled with its scale in
// `sc` (1 for the other precisions), so a linear operation can apply the scale
// to fewer numbers (the 4 link components instead of the 8 NC spinor reals).
template <int NC, int PREC, class T>
__device__ __forceinline__ void load_spinor_raw(const void *base, int nblk, int j, cpx<T> (&s)[4][NC], float &sc)
{
    if constexpr (PREC == kF16) {
        using L = SpinorLayout<NC, PREC>;
        constexpr int NV = L::NVEC;
        const uint4 *p = (const uint4 *)base;
        sc = __ldg((const float *)((const char *)base + L::data_bytes(nblk)) + j);
        float r[8 * NC];
#pragma unroll
        for (int v = 0; v < NV; ++v) halves_to_floats(__ldg(p + vec_index(j, v, NV)), &r[8 * v]);
        values_from_packed<NC>(r, 1.f, s);
    } else {
        sc = 1.f;
        load_spinor<NC, PREC>(base, nblk, j, s);
    }
}

template <int NC, int PREC, class T>
__device__ __forceinline__ void store_spinor(void *base, int nblk, int j, const cpx<T> (&s)[4][NC])
{
    using L = SpinorLayout<NC, PREC>;
    constexpr int NV = L::NVEC;
    if constexpr (PREC == kF64) {
        float4 *p = (float4 *)base;
        float4 w[NV];
        f64_to_vecs<NC>(s, w);
#pragma unroll
        for (int v = 0; v < NV; ++v) p[vec_index(j, v, NV)] = w[v];
    } else if constexpr (PREC == kF32) {
        float4 *p = (float4 *)base;
        float r[8 * NC];
        values_to_packed<NC>(s, r);
#pragma unroll
        for (int v = 0; v < NV; ++v) p[vec_index(j, v, NV)] = make_float4(r[4 * v], r[4 * v + 1], r[4 * v + 2], r[4 * v + 3]);
    } else {
        uint4 *p = (uint4 *)base;
        float *nrm = (float *)((char *)base + L::data_bytes(nblk));
        float f[8 * NC];
        values_to_packed<NC>(s, f);
        float m = 0.f;
#pragma unroll
        for (int k = 0; k < 8 * NC; ++k) m = fmaxf(m, fabsf(f[k]));
        float inv = m > 0.f ? 1.f / m : 0.f;
        nrm[j] = m;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            uint32_t u[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                __half2 h = __floats2half2_rn(f[8 * v + 2 * q] * inv, f[8 * v + 2 * q + 1] * inv);
                u[q] = *reinterpret_cast<uint32_t *>(&h);
            }
            p[vec_index(j, v, NV)] = make_uint4(u[0], u[1], u[2], u[3]);
        }
    }
}

// Decode the NV raw 16-byte vectors of one packed site (plus the FP16 scale)
// into values: the same conversion as load_spinor, for data staged in shared
// memory.
template <int NC, int PREC, class T>
__device__ __forceinline__ void spinor_from_vecs(const uint4 *w, float sc, cpx<T> (&s)[4][NC])
{
    constexpr int NV = SpinorLayout<NC, PREC>::NVEC;
    if constexpr (PREC == kF64) {
        float4 f[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) f[v] = *reinterpret_cast<const float4 *>(&w[v]);
        f64_from_vecs<NC>(f, s);
    } else if constexpr (PREC == kF32) {
        float r[8 * NC];
#pragma unroll
        for (int v = 0; v < NV; ++v) float4_to_floats(*reinterpret_cast<const float4 *>(&w[v]), &r[4 * v]);
        values_from_packed<NC>(r, 1.f, s);
    } else {
        float r[8 * NC];
#pragma unroll
        for (int v = 0; v < NV; ++v) halves_to_floats(w[v], &r[8 * v]);
        values_from_packed<NC>(r, sc, s);
    }
}

// Gauge: quaternion links
template <int PREC> struct GaugeQuat {
    static size_t bytes(int nblk_g)
    {
        size_t per = (PREC == kF64) ? 32 : (PREC == kF32 ? 16 : 8);
        return (size_t)8 * nblk_g * 32 * per;
    }
};

template <int PREC, class T>
__device__ __forceinline__ void load_quat(const void *base, int nblk_g, int p, int mu, int i, T (&a)[4])
{
    size_t slot = (size_t)(p * 4 + mu) * nblk_g + (i >> 5);
    int lane = i & 31;
    if constexpr (PREC == kF64) {
        // (a0.h, a1.h, a2.h, a3.h) then (a0.l, a1.l, a2.l, a3.l)
        const float4 *q = (const float4 *)base;
        float4 hi = __ldg(q + (slot * 2 + 0) * 32 + lane);
        float4 lo = __ldg(q + (slot * 2 + 1) * 32 + lane);
        if constexpr (std::is_same<T, dd>::value) {
            a[0] = dd(hi.x, lo.x); a[1] = dd(hi.y, lo.y); a[2] = dd(hi.z, lo.z); a[3] = dd(hi.w, lo.w);
        } else {
            a[0] = Real<T>::from_double(dd_to_double(dd(hi.x, lo.x)));
            a[1] = Real<T>::from_double(dd_to_double(dd(hi.y, lo.y)));
            a[2] = Real<T>::from_double(dd_to_double(dd(hi.z, lo.z)));
            a[3] = Real<T>::from_double(dd_to_double(dd(hi.w, lo.w)));
        }
    } else if constexpr (PREC == kF32) {
        float4 w = __ldg((const float4 *)base + slot * 32 + lane);
        a[0] = Real<T>::from_float(w.x); a[1] = Real<T>::from_float(w.y);
        a[2] = Real<T>::from_float(w.z); a[3] = Real<T>::from_float(w.w);
    } else {
        uint2 w = __ldg((const uint2 *)base + slot * 32 + lane);
        float2 f0 = __half22float2(*reinterpret_cast<__half2 *>(&w.x));
        float2 f1 = __half22float2(*reinterpret_cast<__half2 *>(&w.y));
        a[0] = Real<T>::from_float(f0.x); a[1] = Real<T>::from_float(f0.y);
        a[2] = Real<T>::from_float(f1.x); a[3] = Real<T>::from_float(f1.y);
    }
}

// store one quaternion link in the packed layout of PREC (from double: pack kernels)
template <int PREC>
__device__ __forceinline__ void store_quat(void *base, int nblk_g, int p, int mu, int i, const double (&a)[4])
{
    size_t slot = (size_t)(p * 4 + mu) * nblk_g + (i >> 5);
    int lane = i & 31;
    if constexpr (PREC == kF64) {
        dd d[4];
        for (int k = 0; k < 4; ++k) d[k] = dd_from_double(a[k]);
        float4 *q = (float4 *)base;
        q[(slot * 2 + 0) * 32 + lane] = make_float4(d[0].h, d[1].h, d[2].h, d[3].h);
        q[(slot * 2 + 1) * 32 + lane] = make_float4(d[0].l, d[1].l, d[2].l, d[3].l);
    } else if constexpr (PREC == kF32) {
        ((float4 *)base)[slot * 32 + lane] = make_float4((float)a[0], (float)a[1], (float)a[2], (float)a[3]);
    } else {
        __half2 h0 = __floats2half2_rn((float)a[0], (float)a[1]);
        __half2 h1 = __floats2half2_rn((float)a[2], (float)a[3]);
        uint2 w;
        w.x = *reinterpret_cast<uint32_t *>(&h0);
        w.y = *reinterpret_cast<uint32_t *>(&h1);
        ((uint2 *)base)[slot * 32 + lane] = w;
    }
}

// quaternion link from its raw vectors (FP64: hi then lo float4; FP32: one
// float4; FP16: the first 8 bytes)
template <int PREC, class T>
__device__ __forceinline__ void quat_from_vecs(const uint4 *w, T (&a)[4])
{
    if constexpr (PREC == kF64) {
        float4 hi = *reinterpret_cast<const float4 *>(&w[0]);
        float4 lo = *reinterpret_cast<const float4 *>(&w[1]);
        if constexpr (std::is_same<T, dd>::value) {
            a[0] = dd(hi.x, lo.x); a[1] = dd(hi.y, lo.y); a[2] = dd(hi.z, lo.z); a[3] = dd(hi.w, lo.w);
        } else {
            a[0] = Real<T>::from_double(dd_to_double(dd(hi.x, lo.x)));
            a[1] = Real<T>::from_double(dd_to_double(dd(hi.y, lo.y)));
            a[2] = Real<T>::from_double(dd_to_double(dd(hi.z, lo.z)));
            a[3] = Real<T>::from_double(dd_to_double(dd(hi.w, lo.w)));
        }
    } else if constexpr (PREC == kF32) {
        float4 f = *reinterpret_cast<const float4 *>(&w[0]);
        a[0] = Real<T>::from_float(f.x); a[1] = Real<T>::from_float(f.y);
        a[2] = Real<T>::from_float(f.z); a[3] = Real<T>::from_float(f.w);
    } else {
        uint32_t x = w[0].x, y = w[0].y;
        float2 f0 = __half22float2(*reinterpret_cast<const __half2 *>(&x));
        float2 f1 = __half22float2(*reinterpret_cast<const __half2 *>(&y));
        a[0] = Real<T>::from_float(f0.x); a[1] = Real<T>::from_float(f0.y);
        a[2] = Real<T>::from_float(f1.x); a[3] = Real<T>::from_float(f1.y);
    }
}

// number of 16-byte staging slots a quaternion link takes
template <int PREC> struct QuatSlots { static constexpr int n = (PREC == kF64) ? 2 : 1; };

// global address of quaternion vector v (FP16: an 8-byte element)
template <int PREC>
__device__ __forceinline__ const void *quat_addr(const void *base, int nblk_g, int p, int mu, int i, int v)
{
    size_t slot = (size_t)(p * 4 + mu) * nblk_g + (i >> 5);
    int lane = i & 31;
    if constexpr (PREC == kF64) return (const uint4 *)base + (slot * 2 + v) * 32 + lane;
    else if constexpr (PREC == kF32) return (const uint4 *)base + slot * 32 + lane;
    else return (const uint2 *)base + slot * 32 + lane;
}

// ---------------------------------------------------------------- async copies
// cp.async global -> shared (Ampere and later, sm_103a included): the copy runs
// in the background; commit_group / wait_group order a thread's own copies.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Bulk (TMA, non-tensor) copies global -> shared completing on an mbarrier
// (sm_90 and later): one thread queues a contiguous copy of `bytes` (a multiple
// of 16, both addresses 16-byte aligned) and the barrier's transaction count
// tells the waiting threads when it has landed.
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    unsigned b = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(b), "r"(count) : "memory");
    // make the initialised barrier visible to the async (TMA) proxy
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_inval(unsigned long long *bar)
{
    unsigned b = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(b) : "memory");
}
// order this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy ones (a bulk copy overwriting data the block has read)
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
// announce `bytes` of transactions on the barrier and arrive (the phase
// completes when the bytes have landed)
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes)
{
    unsigned b = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(b), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void *smem, const void *gmem, unsigned bytes, unsigned long long *bar)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    unsigned b = (unsigned)__cvta_generic_to_shared(bar);
    mbar_arrive_expect_tx(bar, bytes);
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(s),
                 "l"(gmem), "r"(bytes), "r"(b)
                 : "memory");
}
// Wait for phase `parity` of the barrier to complete, for at most about
// `max_cycles` SM clock cycles; false if it did not (the caller records an
// error and must not reuse the destination before a later wait succeeds).
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity, long long max_cycles)
{
    unsigned b = (unsigned)__cvta_generic_to_shared(bar);
    const long long t0 = clock64();
    for (;;) {
        unsigned done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done)
                     : "r"(b), "r"(parity)
                     : "memory");
        if (done) return true;
        if (clock64() - t0 > max_cycles) return false;
    }
}

template <int PREC> struct GaugeMat {
    static size_t bytes(int nblk_g)
    {
        size_t per = (PREC == kF64) ? 8 : (PREC == kF32 ? 4 : 2);
        return (size_t)8 * nblk_g * 32 * 9 * per;
    }
};

template <int PREC, class T>
__device__ __forceinline__ void load_mat(const void *base, int nblk_g, int p, int mu, int i, T (&R)[3][3])
{
    size_t slot = (size_t)(p * 4 + mu) * nblk_g + (i >> 5);
    int lane = i & 31;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
        size_t idx = (slot * 9 + e) * 32 + lane;
        T v;
        if constexpr (PREC == kF64) {
            float2 w = __ldg((const float2 *)base + idx);
            if constexpr (std::is_same<T, dd>::value) v = dd(w.x, w.y);
            else v = Real<T>::from_double(dd_to_double(dd(w.x, w.y)));
        } else if constexpr (PREC == kF32) {
            v = Real<T>::from_float(__ldg((const float *)base + idx));
        } else {
            v = Real<T>::from_float(__half2float(((const __half *)base)[idx]));
        }
        R[e / 3][e % 3] = v;
    }
}

template <int PREC>
__device__ __forceinline__ void store_mat_entry(void *base, int nblk_g, int p, int mu, int i, int e, double v)
{
    size_t slot = (size_t)(p * 4 + mu) * nblk_g + (i >> 5);
    size_t idx = (slot * 9 + e) * 32 + (i & 31);
    if constexpr (PREC == kF64) {
        dd d = dd_from_double(v);
        ((float2 *)base)[idx] = make_float2(d.h, d.l);
    } else if constexpr (PREC == kF32) {
        ((float *)base)[idx] = (float)v;
    } else {
        ((__half *)base)[idx] = __float2half_rn((float)v);
    }
}

// Adjoint link of a unit quaternion: R_bc = (a0^2-|a|^2) d_bc + 2 a_b a_c + 2 a0 eps_bck a_k
__device__ __forceinline__ bool sign_bit(float x) { return (__float_as_uint(x) >> 31) != 0; }
__device__ __forceinline__ bool sign_bit(double x) { return __double_as_longlong(x) < 0; }
__device__ __forceinline__ bool sign_bit(const dd &x) { return sign_bit(x.h); }

// R_ab = 1/2 tr(s_a U s_b U^+) = (a0^2 - |a|^2) d_ab + 2 a_a a_b + 2 a0 e_abc a_c,
// negated when the sign bit of a0 is set: R(q) = R(-q), and the packed
// adjoint links keep that bit clear except on an antiperiodic boundary slice,
// where it carries the factor -1 of the boundary condition
// exact multiplication by a power of two (+-2 here): both parts of a pair scale
__device__ __forceinline__ float scale_pow2(float x, float s) { return x * s; }
__device__ __forceinline__ double scale_pow2(double x, float s) { return x * s; }
__device__ __forceinline__ dd scale_pow2(const dd &x, float s) { return dd(x.h * s, x.l * s); }

template <class T> __device__ __forceinline__ void quat_to_adj(const T (&a)[4], T (&R)[3][3])
{
    // The sign s enters as -w and as the factor 2 s of every product term.
    // Four squares give w = (a0^2 - a2^2) - (a1^2 + a3^2) and the diagonal
    // s w + 2 s a_k^2; the off-diagonal entries come in pairs that share
    // their two products (R_ab and R_ba hold 2 s a_a a_b + and - 2 s a0 a_c),
    // so six products serve the six entries.  The doublings are exact.  The
    // paired adjoint kernels build the same entries two at a time on f32x2
    // lanes with these operations in this order (bit-identical results).
    const bool neg = sign_bit(a[0]);
    const float s2 = neg ? -2.f : 2.f;
    const T sq0 = a[0] * a[0], sq1 = a[1] * a[1], sq2 = a[2] * a[2], sq3 = a[3] * a[3];
    T w = (sq0 - sq2) - (sq1 + sq3);
    if (neg) w = -w;
    R[0][0] = w + scale_pow2(sq1, s2);
    R[1][1] = w + scale_pow2(sq2, s2);
    R[2][2] = w + scale_pow2(sq3, s2);
    const T m12 = scale_pow2(a[1] * a[2], s2), m13 = scale_pow2(a[1] * a[3], s2);
    const T m03 = scale_pow2(a[0] * a[3], s2), m02 = scale_pow2(a[0] * a[2], s2);
    const T m23 = scale_pow2(a[2] * a[3], s2), m01 = scale_pow2(a[0] * a[1], s2);
    R[0][1] = m12 + m03; R[0][2] = m13 - m02;
    R[1][0] = m12 - m03; R[2][0] = m13 + m02;
    R[1][2] = m23 + m01; R[2][1] = m23 - m01;
}

// ---------------------------------------------------------------- colour algebra

// r = U h (DAG = false) or U^+ h (DAG = true), U = a0 + i a.s
template <bool DAG, class T>
__device__ __forceinline__ void su2_mul(const T (&a)[4], const cpx<T> (&h)[2], cpx<T> (&r)[2])
{
    const T a0 = a[0];
    const T a1 = DAG ? -a[1] : a[1], a2 = DAG ? -a[2] : a[2], a3 = DAG ? -a[3] : a[3];
    r[0].re = a0 * h[0].re - a3 * h[0].im + a2 * h[1].re - a1 * h[1].im;
    r[0].im = a0 * h[0].im + a3 * h[0].re + a2 * h[1].im + a1 * h[1].re;
    r[1].re = a0 * h[1].re + a3 * h[1].im - a2 * h[0].re - a1 * h[0].im;
    r[1].im = a0 * h[1].im - a3 * h[1].re - a2 * h[0].im + a1 * h[0].re;
}

// r = R h (DAG = false) or R^T h (real 3x3)
template <bool DAG, class T>
__device__ __forceinline__ void so3_mul(const T (&R)[3][3], const cpx<T> (&h)[3], cpx<T> (&r)[3])
{
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        T m0 = DAG ? R[0][b] : R[b][0], m1 = DAG ? R[1][b] : R[b][1], m2 = DAG ? R[2][b] : R[b][2];
        r[b].re = m0 * h[0].re + m1 * h[1].re + m2 * h[2].re;
        r[b].im = m0 * h[0].im + m1 * h[1].im + m2 * h[2].im;
    }
}

// ---------------------------------------------------------------- spin algebra
// (1 -/+ g_mu) psi = (h, P h) with a 2-spin half spinor h; FWD selects (1 - g_mu).

template <int MU, bool FWD, class T, int NC>
__device__ __forceinline__ void spin_project(const cpx<T> (&s)[4][NC], cpx<T> (&h)[2][NC])
{
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        if constexpr (MU == 0) {
            h[0][c] = FWD ? csub(s[0][c], s[2][c]) : cadd(s[0][c], s[2][c]);
            h[1][c] = FWD ? csub(s[1][c], s[3][c]) : cadd(s[1][c], s[3][c]);
        } else if constexpr (MU == 1) {
            h[0][c] = FWD ? cadd_i(s[0][c], s[3][c]) : csub_i(s[0][c], s[3][c]);
            h[1][c] = FWD ? cadd_i(s[1][c], s[2][c]) : csub_i(s[1][c], s[2][c]);
        } else if constexpr (MU == 2) {
            h[0][c] = FWD ? cadd(s[0][c], s[3][c]) : csub(s[0][c], s[3][c]);
            h[1][c] = FWD ? csub(s[1][c], s[2][c]) : cadd(s[1][c], s[2][c]);
        } else {
            h[0][c] = FWD ? cadd_i(s[0][c], s[2][c]) : csub_i(s[0][c], s[2][c]);
            h[1][c] = FWD ? csub_i(s[1][c], s[3][c]) : cadd_i(s[1][c], s[3][c]);
        }
    }
}

// acc (+)= r, -r, i r or -i r; FIRST: acc holds nothing yet, so assign (the
// first direction of a site saves the additions to zero)
template <bool FIRST, class T> __device__ __forceinline__ cpx<T> acc_add(cpx<T> a, cpx<T> b)
{
    if constexpr (FIRST) return b;
    else return cadd(a, b);
}
template <bool FIRST, class T> __device__ __forceinline__ cpx<T> acc_sub(cpx<T> a, cpx<T> b)
{
    if constexpr (FIRST) return {-b.re, -b.im};
    else return csub(a, b);
}
template <bool FIRST, class T> __device__ __forceinline__ cpx<T> acc_add_i(cpx<T> a, cpx<T> b)
{
    if constexpr (FIRST) return {-b.im, b.re};
    else return cadd_i(a, b);
}
template <bool FIRST, class T> __device__ __forceinline__ cpx<T> acc_sub_i(cpx<T> a, cpx<T> b)
{
    if constexpr (FIRST) return {b.im, -b.re};
    else return csub_i(a, b);
}

// acc += (r, P r): the lower two spins of (1 -/+ g_mu) rebuilt from the upper two
template <int MU, bool FWD, class T, int NC, bool FIRST = false>
__device__ __forceinline__ void spin_accumulate(cpx<T> (&acc)[4][NC], const cpx<T> (&r)[2][NC])
{
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        acc[0][c] = acc_add<FIRST>(acc[0][c], r[0][c]);
        acc[1][c] = acc_add<FIRST>(acc[1][c], r[1][c]);
        if constexpr (MU == 0) {
            if (FWD) { acc[2][c] = acc_sub<FIRST>(acc[2][c], r[0][c]); acc[3][c] = acc_sub<FIRST>(acc[3][c], r[1][c]); }
            else { acc[2][c] = acc_add<FIRST>(acc[2][c], r[0][c]); acc[3][c] = acc_add<FIRST>(acc[3][c], r[1][c]); }
        } else if constexpr (MU == 1) {
            if (FWD) { acc[2][c] = acc_sub_i<FIRST>(acc[2][c], r[1][c]); acc[3][c] = acc_sub_i<FIRST>(acc[3][c], r[0][c]); }
            else { acc[2][c] = acc_add_i<FIRST>(acc[2][c], r[1][c]); acc[3][c] = acc_add_i<FIRST>(acc[3][c], r[0][c]); }
        } else if constexpr (MU == 2) {
            if (FWD) { acc[2][c] = acc_sub<FIRST>(acc[2][c], r[1][c]); acc[3][c] = acc_add<FIRST>(acc[3][c], r[0][c]); }
            else { acc[2][c] = acc_add<FIRST>(acc[2][c], r[1][c]); acc[3][c] = acc_sub<FIRST>(acc[3][c], r[0][c]); }
        } else {
            if (FWD) { acc[2][c] = acc_sub_i<FIRST>(acc[2][c], r[0][c]); acc[3][c] = acc_add_i<FIRST>(acc[3][c], r[1][c]); }
            else { acc[2][c] = acc_add_i<FIRST>(acc[2][c], r[0][c]); acc[3][c] = acc_sub_i<FIRST>(acc[3][c], r[1][c]); }
        }
    }
}

// ---------------------------------------------------------------- reductions

// Deterministic grid reduction of up to 32 per-RHS sums.  Every thread passes
// its value for right-hand side (j & (nrhs-1)); the block's per-RHS sums go to
// partials[blockIdx.x*nrhs + r]; the last block to finish adds the partials in
// block order into sums[r] and returns true (only in that block).
struct RedSlot {
    double *partials;  // >= gridDim.x * nrhs doubles
    unsigned *counter; // zero before the launch; reset by the last block
    // two-level form (nullable): kRedGroup consecutive blocks form a group;
    // the last block of a group to finish sums the group's partials into
    // group_partials[group * nrhs + r] (counted in group_counters[group],
    // zero before the launch, reset), and the last group summer adds the
    // groups.  No block then sums more than kRedGroup blocks' partials.
    unsigned *group_counters; // >= kRedMaxGroups
    double *group_partials;   // >= kRedMaxGroups * nrhs doubles
};
constexpr int kRedGroup = 64, kRedMaxGroups = 64;

__device__ __forceinline__ double warp_sum_strided(double v, int nrhs)
{
    for (int off = 16; off >= nrhs; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// sums[r] = sum over b < nparts of partials[b*nrhs + r], by the whole block.
// Thread t takes right-hand side t % nrhs and every (blockDim/nrhs)-th partial;
// the per-thread sums meet in a fixed tree, so the result does not depend on
// which block runs this.  The partials are read through L2 (ld.cg): other
// blocks wrote them.  Ends with a block barrier; smem >= 32 doubles per warp.
__device__ inline void sum_partials(const double *partials, unsigned nparts, int nrhs, double *sums, double *smem)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int r = threadIdx.x & (nrhs - 1);
    const unsigned step = blockDim.x / nrhs;
    // sixteen independent accumulators keep sixteen L2 loads in flight per
    // thread (a single running sum leaves this one block latency-bound when
    // there are many partials, e.g. 4096 blocks x 32 right-hand sides);
    // combined in a fixed order
    constexpr int K = 16;
    double acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.0;
    unsigned b = threadIdx.x / nrhs;
    for (; b + (K - 1) * step < nparts; b += K * step) {
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] += __ldcg(partials + (size_t)(b + k * step) * nrhs + r);
    }
    for (int k = 0; b < nparts; b += step, ++k) acc[k & (K - 1)] += __ldcg(partials + (size_t)b * nrhs + r);
#pragma unroll
    for (int w = K / 2; w > 0; w >>= 1)
#pragma unroll
        for (int k = 0; k < w; ++k) acc[k] += acc[k + w];
    double s = acc[0];
    s = warp_sum_strided(s, nrhs);
    __syncthreads();
    if (lane < nrhs) smem[warp * 32 + lane] = s;
    __syncthreads();
    if (threadIdx.x < nrhs) {
        double t = 0;
        for (int w = 0; w < nwarps; ++w) t += smem[w * 32 + threadIdx.x];
        sums[threadIdx.x] = t;
    }
    __syncthreads();
}

// The warp stage of a grid reduction in the accumulator's own arithmetic:
// FP32 sums add as floats, double-float sums as pairs on the FP32 pipes (this
// GPU's FP64 unit runs at a small fraction of the FP32 rate, and a reducing
// hop would otherwise convert and shuffle a double on every thread); the
// warp's total becomes a double once.  Lanes r < nrhs return right-hand side
// r's total (the same butterfly order as warp_sum_strided: deterministic).
__device__ __forceinline__ double warp_total(const SqAcc<float> &a, int nrhs)
{
    float v = a.s;
    for (int off = 16; off >= nrhs; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return (double)v;
}
__device__ __forceinline__ double warp_total(const SqAcc<dd> &a, int nrhs)
{
    dd v = a.s;
    for (int off = 16; off >= nrhs; off >>= 1)
        v += dd(__shfl_xor_sync(0xffffffffu, v.h, off), __shfl_xor_sync(0xffffffffu, v.l, off));
    return dd_to_double(v);
}
__device__ __forceinline__ double warp_total(const SqAcc<double> &a, int nrhs)
{
    return warp_sum_strided(a.s, nrhs);
}

// grid_reduce from per-warp totals (lanes r < nrhs hold right-hand side r's)
__device__ inline bool grid_reduce_warped(double v, int nrhs, RedSlot slot, double *sums, double *smem)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    if (lane < nrhs) smem[warp * 32 + lane] = v;
    __syncthreads();
    if (threadIdx.x < nrhs) {
        double s = 0;
        for (int w = 0; w < nwarps; ++w) s += smem[w * 32 + threadIdx.x];
        slot.partials[(size_t)blockIdx.x * nrhs + threadIdx.x] = s;
        // only the writers of the partials order them before the block's
        // count: a fence on every thread would hold each block until its
        // output stores had drained
        __threadfence();
    }
    __shared__ bool last;
    __syncthreads();
    unsigned nparts = gridDim.x;
    const double *parts = slot.partials;
    if (slot.group_counters && gridDim.x > (unsigned)kRedGroup) {
        // first level: the last block of this group sums the group's partials
        const unsigned grp = blockIdx.x / kRedGroup;
        const unsigned first = grp * kRedGroup;
        const unsigned gsize = min((unsigned)kRedGroup, gridDim.x - first);
        if (threadIdx.x == 0) {
            unsigned t = atomicAdd(slot.group_counters + grp, 1u);
            last = (t == gsize - 1);
        }
        __syncthreads();
        if (!last) return false;
        __threadfence();
        sum_partials(slot.partials + (size_t)first * nrhs, gsize, nrhs, sums, smem);
        if (threadIdx.x < nrhs) {
            slot.group_partials[(size_t)grp * nrhs + threadIdx.x] = sums[threadIdx.x];
            __threadfence();
        }
        if (threadIdx.x == 0) slot.group_counters[grp] = 0u;
        __syncthreads();
        nparts = (gridDim.x + kRedGroup - 1) / kRedGroup;
        parts = slot.group_partials;
    }
    if (threadIdx.x == 0) {
        unsigned t = atomicAdd(slot.counter, 1u);
        last = (t == nparts - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    sum_partials(parts, nparts, nrhs, sums, smem);
    if (threadIdx.x == 0) *slot.counter = 0u;
    return true;
}

// Deterministic grid reduction of a value per thread (see RedSlot)
__device__ inline bool grid_reduce(double v, int nrhs, RedSlot slot, double *sums, double *smem /* >= 32*32 */)
{
    return grid_reduce_warped(warp_sum_strided(v, nrhs), nrhs, slot, sums, smem);
}
// ... and of a sum-of-squares accumulator per thread, warp stage in its own arithmetic
template <class T>
__device__ inline bool grid_reduce(const SqAcc<T> &acc, int nrhs, RedSlot slot, double *sums, double *smem)
{
    return grid_reduce_warped(warp_total(acc, nrhs), nrhs, slot, sums, smem);
}

// ---------------------------------------------------------------- solver scalars
constexpr int kMaxRhsSlots = 32;

// offsets (in units of kMaxRhsSlots doubles) of a context's solver scalar block
enum ScalSlot {
    S_RR = 0,      // |r|^2 of the current recurrence
    S_PAP = 1,     // <p, A p> = |Mhat p|^2
    S_ALPHA = 2,
    S_BETA = 3,
    S_BB = 4,      // |b|^2
    S_STOP = 5,    // tol^2 |b|^2
    S_ACTIVE = 6,  // 1.0 while the RHS is iterating
    S_RMAX = 7,    // max |r|^2 since the last reliable update
    S_RROLD = 8,   // |r|^2 before the current iteration
    S_OUT = 9,     // generic reduction output
    S_FLAGS = 10,  // [0] all done, [1] reliable-update gate, [2] NaN/Inf seen, [3] iterations,
                   // [4] reliable updates, [5] device-loop passes, [6] device error (a
                   // bulk copy that did not land in time), [7] source out of range,
                   // [8] S_OUT holds the true FP64 residuals of the current x (the
                   // last scalar update was a reliable update's), [9] / [10] the
                   // open reliable update is of the FP32 / FP64 tier
    S_DELTA2 = 11, // [0] reliable-update threshold delta^2, [1] tol^2, [2] maxiter (<= 0: none),
                   // [3] FP32-tier threshold delta_mid^2 (0: every update is an FP64 one)
    S_SCALE = 12,  // per-RHS power of two that brings the source's largest component into [0.5, 1)
    S_BMAX = 13,   // per-RHS largest |component| of the source, as the bits of a float (32 unsigned)
    S_RREF = 14,   // |r|^2 of the last FP64 residual (the FP32 tier's reference)
    S_NSLOTS = 15
};
constexpr int F_DONE = 0, F_GATE = 1, F_NUMERIC = 2, F_ITERS = 3, F_NRELIABLE = 4, F_BODY = 5, F_DEVERR = 6,
              F_RANGE = 7, F_TRUERES = 8, F_TIER1 = 9, F_TIER2 = 10;

enum FinishMode {
    kFinNone = 0,
    kFinStore = 1,      // scal[S_OUT] = sums
    kFinAlpha = 2,      // pAp = sums; alpha = active ? rr / pAp : 0
    kFinBeta = 3,       // rr_new = sums; beta; converged RHS stop
    kFinBetaMixed = 4,  // as kFinBeta, but convergence and small residuals open the reliable-update gate
    kFinResidual = 5,   // true FP64 residual of a reliable update: restart bookkeeping, close the gate
    kFinInit = 6,       // |r0|^2: rr = rmax = rrold = sums, a RHS is active while rr > stop
    kFinBB = 7,         // |b|^2: bb = sums, stop = tol^2 bb (tol^2 in scal[S_DELTA2][1])
    kFinMid = 8         // residual of an FP32-tier reliable update: restart bookkeeping (no stop), close the gate
};

__device__ __forceinline__ double &sc(double *scal, int slot, int r) { return scal[slot * kMaxRhsSlots + r]; }

// Scalar updates run by the last block of a grid reduction (threads 0..nrhs-1
// hold one right-hand side each); afterwards thread 0 refreshes the flags.
__device__ inline void finish_reduction(int mode, const double *sums, int nrhs, double *scal)
{
    const int r = threadIdx.x;
    if (r < nrhs) {
        double v = sums[r];
        bool bad = !isfinite(v);
        bool act = sc(scal, S_ACTIVE, r) != 0.0;
        switch (mode) {
        case kFinStore:
            sc(scal, S_OUT, r) = v;
            break;
        case kFinAlpha:
            sc(scal, S_PAP, r) = v;
            sc(scal, S_ALPHA, r) = (act && v > 0.0) ? sc(scal, S_RR, r) / v : 0.0;
            break;
        case kFinBeta:
        case kFinBetaMixed: {
            double rr = sc(scal, S_RR, r);
            sc(scal, S_RROLD, r) = rr;
            if (act) {
                sc(scal, S_BETA, r) = v / rr;
                sc(scal, S_RR, r) = v;
                if (mode == kFinBeta) {
                    if (v <= sc(scal, S_STOP, r)) sc(scal, S_ACTIVE, r) = 0.0;
                } else {
                    double rmax = fmax(sc(scal, S_RMAX, r), v);
                    sc(scal, S_RMAX, r) = rmax;
                    const bool conv = v <= sc(scal, S_STOP, r);
                    if (conv || v < sc(scal, S_DELTA2, 0) * rmax) {
                        sc(scal, S_FLAGS, F_GATE) = 1.0;
                        // the FP64 tier when the FP32 tier is off, at convergence, or
                        // once |r| fell by delta_mid since the last FP64 residual
                        const double dm = sc(scal, S_DELTA2, 3);
                        if (dm == 0.0 || conv || v < dm * sc(scal, S_RREF, r)) sc(scal, S_FLAGS, F_TIER2) = 1.0;
                    }
                }
            } else {
                sc(scal, S_BETA, r) = 0.0;
            }
            break;
        }
        case kFinInit:
            sc(scal, S_RR, r) = v;
            sc(scal, S_RMAX, r) = v;
            sc(scal, S_RROLD, r) = v;
            sc(scal, S_RREF, r) = v;
            sc(scal, S_ACTIVE, r) = (v > sc(scal, S_STOP, r)) ? 1.0 : 0.0;
            break;
        case kFinBB:
            sc(scal, S_BB, r) = v;
            sc(scal, S_STOP, r) = sc(scal, S_DELTA2, 1) * v;
            break;
        case kFinResidual:
            if (act) {
                sc(scal, S_BETA, r) = v / sc(scal, S_RROLD, r);
                sc(scal, S_RR, r) = v;
                sc(scal, S_RMAX, r) = v;
                if (v <= sc(scal, S_STOP, r)) sc(scal, S_ACTIVE, r) = 0.0;
            } else {
                sc(scal, S_BETA, r) = 0.0;
            }
            sc(scal, S_OUT, r) = v;
            sc(scal, S_RREF, r) = v;
            break;
        case kFinMid:
            // r = r_ref - A_32 dx is accurate to FP32 relative to r_ref only: it
            // restarts the recurrence but stops no right-hand side
            if (act) {
                sc(scal, S_BETA, r) = v / sc(scal, S_RROLD, r);
                sc(scal, S_RR, r) = v;
                sc(scal, S_RMAX, r) = v;
            } else {
                sc(scal, S_BETA, r) = 0.0;
            }
            break;
        default:
            break;
        }
        if (bad && mode != kFinStore) sc(scal, S_FLAGS, F_NUMERIC) = 1.0;
    }
    __syncthreads();
    if (threadIdx.x == 0 && mode != kFinStore && mode != kFinBB) {
        bool all_done = true;
        for (int k = 0; k < nrhs; ++k) all_done = all_done && (sc(scal, S_ACTIVE, k) == 0.0);
        if (sc(scal, S_FLAGS, F_NUMERIC) != 0.0) all_done = true;
        if (mode == kFinBeta || mode == kFinBetaMixed) {
            // the iteration cap also stops the recurrence (work already queued skips)
            const double it = sc(scal, S_FLAGS, F_ITERS) + 1.0, cap = sc(scal, S_DELTA2, 2);
            sc(scal, S_FLAGS, F_ITERS) = it;
            if (cap > 0.0 && it >= cap) all_done = true;
        }
        sc(scal, S_FLAGS, F_DONE) = all_done ? 1.0 : 0.0;
        if (mode == kFinResidual) {
            sc(scal, S_FLAGS, F_GATE) = 0.0;
            sc(scal, S_FLAGS, F_TIER1) = 0.0;
            sc(scal, S_FLAGS, F_TIER2) = 0.0;
            sc(scal, S_FLAGS, F_NRELIABLE) += 1.0;
            // x_lo was folded into x and S_OUT = |b - A x|^2: a loop that stops
            // here needs no further true-residual computation
            sc(scal, S_FLAGS, F_TRUERES) = 1.0;
        } else if (mode == kFinMid) {
            sc(scal, S_FLAGS, F_GATE) = 0.0;
            sc(scal, S_FLAGS, F_TIER1) = 0.0;
            sc(scal, S_FLAGS, F_TRUERES) = 0.0;
        } else if (mode == kFinBeta || mode == kFinBetaMixed || mode == kFinInit) {
            sc(scal, S_FLAGS, F_TRUERES) = 0.0; // x (or x_lo) moved since
        }
        // an open gate is of exactly one tier
        if (mode == kFinBetaMixed && sc(scal, S_FLAGS, F_GATE) != 0.0)
            sc(scal, S_FLAGS, F_TIER1) = sc(scal, S_FLAGS, F_TIER2) != 0.0 ? 0.0 : 1.0;
    }
}

} // namespace hr
