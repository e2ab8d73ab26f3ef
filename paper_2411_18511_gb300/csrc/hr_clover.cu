// hr_clover.cu -- the clover and exponential-clover site terms
// (arXiv:2411.18511 Sec. 2.2): building the packed field once per gauge field
// (A and A^-1, or (4+m0) exp(+-c_sw C/(4+m0)), on both parities), converting it
// to FP32 for the mixed-precision operators, applying it on one parity, and
// the full and even-odd operators with the site term.  The products inside the
// hop (A_ee on the aux term, A_oo^-1 on the result) run in the hop epilogue
// (hr_hop_dev.cuh), so every hop kernel variant carries them.
//
// Build (native FP64: a precomputation, not the hot path).  Per site x:
//   Q_mn   the four leaves of the (mu, nu) plane from x, mu-first,
//   F_mn = (Q_mn - Q_mn^+) / 8, B_l = e_jkl F_jk / 2 (B_1 = F_23, B_2 = F_31, B_3 = F_12),
//   in the chiral basis s_0k = diag(-s_k, s_k) and s_jk = -e_jkl diag(s_l, s_l), so
//   C = (i/4) sum s_mn F_mn = diag(C+, C-),
//   C+ = sum_l s_l (x) (-(i/2)(F_0l + B_l)),   C- = sum_l s_l (x) ((i/2)(F_0l - B_l)),
//   clover:      A = (4+m0) + c_sw C,            A^-1 by Gauss-Jordan elimination,
//   exponential: A = (4+m0) exp(c_sw C/(4+m0)),  A^-1 = exp(-c_sw C/(4+m0)) / (4+m0),
// the exponential by scaling and squaring of a degree-16 Taylor polynomial
// (the argument is scaled below 1/2 in the 1-norm: truncation < 1e-19).
// Storing the explicit inverse instead of LDL factors: the same n^2 reals, and
// a matrix-vector product has no sequential dependency chain.
#include <cmath>

#include "hr_clover.cuh"
#include "hr_clover_leaf.cuh"
#include "hr_eigh.cuh"
#include "hr_host.h"

using namespace hr;

namespace {

struct zc {
    double re, im;
};
__device__ __forceinline__ zc zadd(zc a, zc b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ zc zsub(zc a, zc b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ zc zmul(zc a, zc b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ zc zconj(zc a) { return {a.re, -a.im}; }
__device__ __forceinline__ zc zscale(double s, zc a) { return {s * a.re, s * a.im}; }

template <int NC> struct CM {
    zc m[NC][NC];
};

// U_mu(x) as a colour matrix from the canonical quaternion (fundamental
// 2x2, or the real adjoint R_ab = 1/2 tr(s_a U s_b U^+))
template <int NC> __device__ CM<NC> link_mat(const double *can, long long V, int mu, long long x)
{
    const double *q = can + ((long long)mu * V + x) * 4;
    const double a0 = q[0], a1 = q[1], a2 = q[2], a3 = q[3];
    CM<NC> U;
    if constexpr (NC == 2) {
        U.m[0][0] = {a0, a3};
        U.m[0][1] = {a2, a1};
        U.m[1][0] = {-a2, a1};
        U.m[1][1] = {a0, -a3};
    } else {
        const double w = a0 * a0 - (a1 * a1 + a2 * a2 + a3 * a3);
        const double a[3] = {a1, a2, a3};
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) U.m[r][c] = {2.0 * a[r] * a[c] + (r == c ? w : 0.0), 0.0};
        U.m[0][1].re += 2.0 * a0 * a3;
        U.m[0][2].re -= 2.0 * a0 * a2;
        U.m[1][0].re -= 2.0 * a0 * a3;
        U.m[1][2].re += 2.0 * a0 * a1;
        U.m[2][0].re += 2.0 * a0 * a2;
        U.m[2][1].re -= 2.0 * a0 * a1;
    }
    return U;
}

// A B, with either factor optionally daggered
template <int NC> __device__ CM<NC> cmul(const CM<NC> &A, bool da, const CM<NC> &B, bool db)
{
    CM<NC> C;
    for (int r = 0; r < NC; ++r)
        for (int c = 0; c < NC; ++c) {
            zc s = {0.0, 0.0};
            for (int k = 0; k < NC; ++k) {
                const zc a = da ? zconj(A.m[k][r]) : A.m[r][k];
                const zc b = db ? zconj(B.m[c][k]) : B.m[k][c];
                s = zadd(s, zmul(a, b));
            }
            C.m[r][c] = s;
        }
    return C;
}

__device__ long long lex_of(const Geom &g, const int (&x)[4])
{
    return (((long long)x[0] * g.d[1] + x[1]) * g.d[2] + x[2]) * g.d[3] + x[3];
}
// the site x + s1 m1 + s2 m2 (periodic; s = 0 leaves a direction alone)
__device__ long long nb(const Geom &g, const int (&x)[4], int m1, int s1, int m2 = 0, int s2 = 0)
{
    int y[4] = {x[0], x[1], x[2], x[3]};
    y[m1] = (y[m1] + s1 + g.d[m1]) % g.d[m1];
    y[m2] = (y[m2] + s2 + g.d[m2]) % g.d[m2];
    return lex_of(g, y);
}

// F_mn(x) = (Q_mn - Q_mn^+)/8 from the four leaves that start at x
template <int NC> __device__ CM<NC> field_strength(const Geom &g, const double *can, const int (&x)[4], int mu, int nu)
{
    const long long V = 2LL * g.vh;
    const long long x0 = lex_of(g, x);
    const long long xpm = nb(g, x, mu, 1), xpn = nb(g, x, nu, 1), xmm = nb(g, x, mu, -1), xmn = nb(g, x, nu, -1);
    const long long xmm_pn = nb(g, x, mu, -1, nu, 1), xmm_mn = nb(g, x, mu, -1, nu, -1), xmn_pm = nb(g, x, nu, -1, mu, 1);
    auto U = [&](int d, long long s) { return link_mat<NC>(can, V, d, s); };
    // U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+
    CM<NC> Q = cmul(cmul(U(mu, x0), false, U(nu, xpm), false), false, cmul(U(nu, x0), false, U(mu, xpn), false), true);
    // U_nu(x) U_mu(x-mu+nu)^+ U_nu(x-mu)^+ U_mu(x-mu)
    CM<NC> t = cmul(cmul(U(nu, x0), false, U(mu, xmm_pn), true), false, cmul(U(nu, xmm), true, U(mu, xmm), false), false);
    for (int r = 0; r < NC; ++r)
        for (int c = 0; c < NC; ++c) Q.m[r][c] = zadd(Q.m[r][c], t.m[r][c]);
    // U_mu(x-mu)^+ U_nu(x-mu-nu)^+ U_mu(x-mu-nu) U_nu(x-nu)
    t = cmul(cmul(U(nu, xmm_mn), false, U(mu, xmm), false), true, cmul(U(mu, xmm_mn), false, U(nu, xmn), false), false);
    for (int r = 0; r < NC; ++r)
        for (int c = 0; c < NC; ++c) Q.m[r][c] = zadd(Q.m[r][c], t.m[r][c]);
    // U_nu(x-nu)^+ U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^+
    t = cmul(cmul(U(nu, xmn), true, U(mu, xmn), false), false, cmul(U(mu, x0), false, U(nu, xmn_pm), true), true);
    for (int r = 0; r < NC; ++r)
        for (int c = 0; c < NC; ++c) Q.m[r][c] = zadd(Q.m[r][c], t.m[r][c]);
    CM<NC> F;
    for (int r = 0; r < NC; ++r)
        for (int c = 0; c < NC; ++c) F.m[r][c] = zscale(0.125, zsub(Q.m[r][c], zconj(Q.m[c][r])));
    return F;
}

template <int N> struct ZM {
    zc m[N][N];
};

template <int N> __device__ ZM<N> zmm(const ZM<N> &A, const ZM<N> &B)
{
    ZM<N> C;
#pragma unroll 1
    for (int r = 0; r < N; ++r)
        for (int c = 0; c < N; ++c) {
            zc s = {0.0, 0.0};
            for (int k = 0; k < N; ++k) s = zadd(s, zmul(A.m[r][k], B.m[k][c]));
            C.m[r][c] = s;
        }
    return C;
}

// exp(X) by scaling and squaring of the degree-16 Taylor polynomial
template <int N> __device__ ZM<N> expm(ZM<N> X)
{
    double nrm = 0.0;
    for (int c = 0; c < N; ++c) {
        double s = 0.0;
        for (int r = 0; r < N; ++r) s += hypot(X.m[r][c].re, X.m[r][c].im);
        nrm = fmax(nrm, s);
    }
    int sq = 0;
    while (nrm > 0.5 && sq < 60) {
        nrm *= 0.5;
        ++sq;
    }
    const double sc = ldexp(1.0, -sq);
    for (int r = 0; r < N; ++r)
        for (int c = 0; c < N; ++c) X.m[r][c] = zscale(sc, X.m[r][c]);
    // Horner: E = 1 + X (1 + X/2 (1 + X/3 (... (1 + X/16))))
    ZM<N> E;
    for (int r = 0; r < N; ++r)
        for (int c = 0; c < N; ++c) E.m[r][c] = {r == c ? 1.0 : 0.0, 0.0};
#pragma unroll 1
    for (int k = 16; k >= 1; --k) {
        ZM<N> T = zmm(X, E);
        for (int r = 0; r < N; ++r)
            for (int c = 0; c < N; ++c) E.m[r][c] = zadd(zscale(1.0 / k, T.m[r][c]), {r == c ? 1.0 : 0.0, 0.0});
    }
#pragma unroll 1
    for (int k = 0; k < sq; ++k) E = zmm(E, E);
    return E;
}

// A^-1 by Gauss-Jordan elimination with partial pivoting (false if singular)
template <int N> __device__ bool inverse(ZM<N> A, ZM<N> &I)
{
    for (int r = 0; r < N; ++r)
        for (int c = 0; c < N; ++c) I.m[r][c] = {r == c ? 1.0 : 0.0, 0.0};
#pragma unroll 1
    for (int k = 0; k < N; ++k) {
        int piv = k;
        double best = -1.0;
        for (int r = k; r < N; ++r) {
            const double m = A.m[r][k].re * A.m[r][k].re + A.m[r][k].im * A.m[r][k].im;
            if (m > best) {
                best = m;
                piv = r;
            }
        }
        if (!(best > 0.0)) return false;
        if (piv != k)
            for (int c = 0; c < N; ++c) {
                zc t = A.m[k][c];
                A.m[k][c] = A.m[piv][c];
                A.m[piv][c] = t;
                t = I.m[k][c];
                I.m[k][c] = I.m[piv][c];
                I.m[piv][c] = t;
            }
        const zc p = A.m[k][k];
        const double pn = p.re * p.re + p.im * p.im;
        const zc pinv = {p.re / pn, -p.im / pn};
        for (int c = 0; c < N; ++c) {
            A.m[k][c] = zmul(A.m[k][c], pinv);
            I.m[k][c] = zmul(I.m[k][c], pinv);
        }
        for (int r = 0; r < N; ++r) {
            if (r == k) continue;
            const zc f = A.m[r][k];
            for (int c = 0; c < N; ++c) {
                A.m[r][c] = zsub(A.m[r][c], zmul(f, A.m[k][c]));
                I.m[r][c] = zsub(I.m[r][c], zmul(f, I.m[k][c]));
            }
        }
    }
    return true;
}

// the n^2 reals of a Hermitian block (diagonal, then the upper triangle as re, im)
template <int N> __device__ void block_reals(const ZM<N> &M, double *out)
{
    int r = 0;
    for (int k = 0; k < N; ++k) out[r++] = M.m[k][k].re;
    for (int p = 0; p < N; ++p)
        for (int q = p + 1; q < N; ++q) {
            out[r++] = M.m[p][q].re;
            out[r++] = M.m[p][q].im;
        }
}

template <int NC, int CP> __device__ void store_site(void *half, int i, const double *reals)
{
    using L = CloverLayout<NC, CP>;
    float4 *base = (float4 *)half;
#pragma unroll 1
    for (int v = 0; v < L::NVEC; ++v) {
        float4 w;
        if constexpr (CP == kF64) {
            const double a = reals[2 * v], b = reals[2 * v + 1];
            const float ah = (float)a, bh = (float)b;
            w = make_float4(ah, (float)(a - (double)ah), bh, (float)(b - (double)bh));
        } else {
            w = make_float4((float)reals[4 * v], (float)reals[4 * v + 1], (float)reals[4 * v + 2],
                            (float)reals[4 * v + 3]);
        }
        base[((size_t)(i >> 5) * L::NVEC + v) * 32 + (i & 31)] = w;
    }
}

struct BuildArgs {
    Geom g;
    const double *can;
    double m0, csw;
    int kind;
    void *half[4]; // A even, A odd, A^-1 even, A^-1 odd
    unsigned *bad; // set when an A is singular
};

// one thread per lexicographic site
template <int NC, int CP> __global__ void __launch_bounds__(64) k_clover_build(BuildArgs B)
{
    constexpr int N = 2 * NC;
    const Geom &g = B.g;
    const long long V = 2LL * g.vh;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= V) return;
    int x[4];
    long long r = t;
    for (int k = 3; k >= 0; --k) {
        x[k] = (int)(r % g.d[k]);
        r /= g.d[k];
    }
    const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
    const int i = (int)(t >> 1);
    // F_mn for the six planes
    CM<NC> F01 = field_strength<NC>(g, B.can, x, 0, 1), F02 = field_strength<NC>(g, B.can, x, 0, 2),
           F03 = field_strength<NC>(g, B.can, x, 0, 3), F12 = field_strength<NC>(g, B.can, x, 1, 2),
           F13 = field_strength<NC>(g, B.can, x, 1, 3), F23 = field_strength<NC>(g, B.can, x, 2, 3);
    const CM<NC> *E[3] = {&F01, &F02, &F03};
    const double a = 4.0 + B.m0;
    double reals[2][2 * N * N]; // [forward / inverse][both blocks]
#pragma unroll 1
    for (int b = 0; b < 2; ++b) {
        // G_l = -(i/2)(F_0l + B_l) (upper block) or (i/2)(F_0l - B_l) (lower)
        ZM<N> C;
        for (int rr = 0; rr < N; ++rr)
            for (int cc = 0; cc < N; ++cc) C.m[rr][cc] = {0.0, 0.0};
        for (int l = 0; l < 3; ++l) {
            const CM<NC> &Bm = l == 0 ? F23 : l == 1 ? F13 : F12;
            const double sB = l == 1 ? -1.0 : 1.0; // B_2 = F_31 = -F_13
            for (int c = 0; c < NC; ++c)
                for (int d = 0; d < NC; ++d) {
                    const zc f = E[l]->m[c][d], bb = zscale(sB, Bm.m[c][d]);
                    const zc s = b == 0 ? zadd(f, bb) : zsub(f, bb);
                    // times -(i/2) or +(i/2)
                    const double h = b == 0 ? -0.5 : 0.5;
                    const zc G = {-h * s.im, h * s.re};
                    // s_l (x) G: s_1 = [[0,1],[1,0]], s_2 = [[0,-i],[i,0]], s_3 = diag(1,-1)
                    if (l == 0) {
                        C.m[c][NC + d] = zadd(C.m[c][NC + d], G);
                        C.m[NC + c][d] = zadd(C.m[NC + c][d], G);
                    } else if (l == 1) {
                        C.m[c][NC + d] = zadd(C.m[c][NC + d], {G.im, -G.re});  // -i G
                        C.m[NC + c][d] = zadd(C.m[NC + c][d], {-G.im, G.re});  // +i G
                    } else {
                        C.m[c][d] = zadd(C.m[c][d], G);
                        C.m[NC + c][NC + d] = zsub(C.m[NC + c][NC + d], G);
                    }
                }
        }
        ZM<N> A, Ai;
        if (B.kind == HR_CLOVER_EXP) {
            ZM<N> X = C, Y = C;
            for (int rr = 0; rr < N; ++rr)
                for (int cc = 0; cc < N; ++cc) {
                    X.m[rr][cc] = zscale(B.csw / a, C.m[rr][cc]);
                    Y.m[rr][cc] = zscale(-B.csw / a, C.m[rr][cc]);
                }
            A = expm(X);
            Ai = expm(Y);
            for (int rr = 0; rr < N; ++rr)
                for (int cc = 0; cc < N; ++cc) {
                    A.m[rr][cc] = zscale(a, A.m[rr][cc]);
                    Ai.m[rr][cc] = zscale(1.0 / a, Ai.m[rr][cc]);
                }
        } else {
            for (int rr = 0; rr < N; ++rr)
                for (int cc = 0; cc < N; ++cc)
                    A.m[rr][cc] = zadd(zscale(B.csw, C.m[rr][cc]), {rr == cc ? a : 0.0, 0.0});
            if (!inverse(A, Ai)) atomicExch(B.bad, 1u);
        }
        block_reals(A, &reals[0][b * N * N]);
        block_reals(Ai, &reals[1][b * N * N]);
    }
    store_site<NC, CP>(B.half[p], i, reals[0]);
    store_site<NC, CP>(B.half[2 + p], i, reals[1]);
}

// FP64 -> FP32 field, one thread per FP32 vector
template <int NC> __global__ void k_clover_to_f32(int nvec_total, const float4 *src, float4 *dst)
{
    using L64 = CloverLayout<NC, kF64>;
    using L32 = CloverLayout<NC, kF32>;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nvec_total) return;
    const int lane = t & 31, v = (t >> 5) % L32::NVEC, blk = (t >> 5) / L32::NVEC;
    const float4 a = src[((size_t)blk * L64::NVEC + 2 * v) * 32 + lane];
    const float4 b = src[((size_t)blk * L64::NVEC + 2 * v + 1) * 32 + lane];
    dst[((size_t)blk * L32::NVEC + v) * 32 + lane] = make_float4(a.x + a.y, a.z + a.w, b.x + b.y, b.z + b.w);
}

// out = A in (or A^-1 in) on the sites of one parity (every right-hand side)
template <int NC, int PREC> __global__ void k_clover_apply(Geom g, const void *half, const void *in, void *out)
{
    using T = typename PrecTraits<PREC>::T;
    const int nv = g.vh << g.lrhs;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nv; j += gridDim.x * blockDim.x) {
        cpx<T> v[4][NC];
        load_spinor<NC, PREC>(in, g.nblk_s, j, v);
        clover_apply<clover_prec(PREC)>(half, j >> g.lrhs, v);
        store_spinor<NC, PREC>(out, g.nblk_s, j, v);
    }
}

bool valid_clover_prec(int prec) { return prec == kF64 || prec == kF32; }

} // namespace

namespace hr {

size_t clover_half_bytes(const Geom &g, int rep, int cp)
{
    if (rep_nc(rep) == 2) return cp == kF64 ? CloverLayout<2, kF64>::half_bytes(g.nblk_g) : CloverLayout<2, kF32>::half_bytes(g.nblk_g);
    return cp == kF64 ? CloverLayout<3, kF64>::half_bytes(g.nblk_g) : CloverLayout<3, kF32>::half_bytes(g.nblk_g);
}

const void *clover_half(const void *base, const Geom &g, int rep, int cp, bool inverse, int parity)
{
    if (!base) return nullptr;
    return (const char *)base + (size_t)((inverse ? 2 : 0) + parity) * clover_half_bytes(g, rep, cp);
}

hr_status clover_convert_f32(hr_ctx *ctx, const Geom &g, int rep, const void *src, void *dst, cudaStream_t s)
{
    const int nc = rep_nc(rep);
    const size_t h64 = clover_half_bytes(g, rep, kF64), h32 = clover_half_bytes(g, rep, kF32);
    const int nvec = g.nblk_g * 32 * (nc == 2 ? CloverLayout<2, kF32>::NVEC : CloverLayout<3, kF32>::NVEC);
    const int bs = 256, grid = (nvec + bs - 1) / bs;
    for (int h = 0; h < 4; ++h) {
        const float4 *a = (const float4 *)((const char *)src + h * h64);
        float4 *b = (float4 *)((char *)dst + h * h32);
        if (nc == 2) k_clover_to_f32<2><<<grid, bs, 0, s>>>(nvec, a, b);
        else k_clover_to_f32<3><<<grid, bs, 0, s>>>(nvec, a, b);
    }
    return check_launch(ctx, "clover convert");
}

hr_status clover_apply_half(hr_ctx *ctx, const Geom &g, int rep, int prec, const void *half, const void *in,
                            void *out, cudaStream_t s)
{
    const long long nv = (long long)g.vh << g.lrhs;
    const int bs = 128, grid = grid_for(nv, bs, 1 << 30);
    const bool three = rep_nc(rep) == 3;
    switch (prec) {
    case kF64:
        if (three) k_clover_apply<3, kF64><<<grid, bs, 0, s>>>(g, half, in, out);
        else k_clover_apply<2, kF64><<<grid, bs, 0, s>>>(g, half, in, out);
        break;
    case kF32:
        if (three) k_clover_apply<3, kF32><<<grid, bs, 0, s>>>(g, half, in, out);
        else k_clover_apply<2, kF32><<<grid, bs, 0, s>>>(g, half, in, out);
        break;
    default:
        if (three) k_clover_apply<3, kF16><<<grid, bs, 0, s>>>(g, half, in, out);
        else k_clover_apply<2, kF16><<<grid, bs, 0, s>>>(g, half, in, out);
        break;
    }
    return check_launch(ctx, "clover apply");
}

} // namespace hr

extern "C" {

size_t hr_clover_packed_bytes(hr_lattice lat, hr_rep rep, hr_prec prec)
{
    if (!valid_rep(rep) || !valid_clover_prec(prec) || hr_gauge_packed_bytes(lat, rep, prec) == 0) return 0;
    return 4 * clover_half_bytes(make_geom(lat, 1), rep, prec);
}

hr_status hr_clover_build(hr_ctx *ctx, hr_lattice lat, hr_rep rep, hr_prec prec, hr_clover_kind kind, double m0,
                          double c_sw, const double *canonical, void *clover, hr_stream stream)
{
    if (!ctx) return HR_ERR_INVALID_ARG;
    if (!valid_rep(rep)) return set_error(ctx, HR_ERR_INVALID_ARG, "bad rep");
    if (!valid_clover_prec(prec)) return set_error(ctx, HR_ERR_UNSUPPORTED, "clover fields are FP64 or FP32");
    if (kind != HR_CLOVER_SW && kind != HR_CLOVER_EXP) return set_error(ctx, HR_ERR_INVALID_ARG, "bad clover kind");
    hr_status st = validate_lattice(ctx, lat, 1);
    if (st) return st;
    st = check_buffers(ctx, {clover}, {canonical});
    if (st) return st;
    if (!(4.0 + m0 != 0.0) || !std::isfinite(m0) || !std::isfinite(c_sw))
        return set_error(ctx, HR_ERR_INVALID_ARG, "4 + m0 must be nonzero and finite, c_sw finite");
    const Geom g = make_geom(lat, 1);
    cudaStream_t s = (cudaStream_t)stream;
    BuildArgs B;
    B.g = g;
    B.can = canonical;
    B.m0 = m0;
    B.csw = c_sw;
    B.kind = kind;
    for (int h = 0; h < 4; ++h) B.half[h] = (void *)clover_half(clover, g, rep, prec, h >= 2, h & 1);
    B.bad = ctx->d_counters + C_STATUS;
    cudaError_t e = cudaMemsetAsync(B.bad, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return set_error(ctx, HR_ERR_CUDA, "status reset: %s", cudaGetErrorString(e));
    const long long V = 2LL * g.vh;
    const int bs = 64, grid = (int)((V + bs - 1) / bs);
    const bool three = rep_nc(rep) == 3;
    if (prec == kF64) {
        if (three) k_clover_build<3, kF64><<<grid, bs, 0, s>>>(B);
        else k_clover_build<2, kF64><<<grid, bs, 0, s>>>(B);
    } else {
        if (three) k_clover_build<3, kF32><<<grid, bs, 0, s>>>(B);
        else k_clover_build<2, kF32><<<grid, bs, 0, s>>>(B);
    }
    st = check_launch(ctx, "clover build");
    if (st) return st;
    unsigned bad = 0;
    e = cudaMemcpyAsync(&bad, B.bad, sizeof bad, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_error(ctx, HR_ERR_CUDA, "clover build status: %s", cudaGetErrorString(e));
    if (bad) return set_error(ctx, HR_ERR_NUMERIC, "a clover site block is singular (no inverse)");
    return HR_OK;
}

hr_status hr_clover_apply(hr_ctx *ctx, hr_lattice lat, hr_rep rep, hr_prec prec, hr_parity parity, int inverse,
                          int n_rhs, const void *clover, const void *in, void *out, hr_stream stream)
{
    if (!ctx) return HR_ERR_INVALID_ARG;
    if (!valid_rep(rep) || !valid_prec(prec)) return set_error(ctx, HR_ERR_INVALID_ARG, "bad rep/prec");
    if (parity != HR_EVEN && parity != HR_ODD) return set_error(ctx, HR_ERR_INVALID_ARG, "parity HR_EVEN or HR_ODD");
    hr_status st = validate_lattice(ctx, lat, n_rhs);
    if (st) return st;
    st = check_buffers(ctx, {clover, in, out});
    if (st) return st;
    const Geom g = make_geom(lat, n_rhs);
    const Geom g1 = make_geom(lat, 1);
    const void *half = clover_half(clover, g1, rep, clover_prec(prec), inverse != 0, parity);
    return clover_apply_half(ctx, g, rep, prec, half, in, out, (cudaStream_t)stream);
}

hr_status hr_dirac_apply_clover(hr_ctx *ctx, hr_lattice lat, hr_rep rep, hr_prec prec, const void *gauge,
                                const void *clover, const void *in, void *out, hr_stream stream)
{
    if (!ctx) return HR_ERR_INVALID_ARG;
    if (!valid_rep(rep) || !valid_prec(prec)) return set_error(ctx, HR_ERR_INVALID_ARG, "bad rep/prec");
    hr_status st = validate_lattice(ctx, lat, 1);
    if (st) return st;
    st = check_buffers(ctx, {gauge, clover, in, out});
    if (st) return st;
    if (in == out) return set_error(ctx, HR_ERR_INVALID_ARG, "in and out must not alias");
    const Geom g = make_geom(lat, 1);
    const size_t half = spinor_half_bytes(g, rep, prec);
    cudaStream_t s = (cudaStream_t)stream;
    // out_p = A_pp in_p - 1/2 H_{p,1-p} in_{1-p}: one hop per parity, A on the aux term
    for (int p = 0; p < 2; ++p) {
        HopLaunch L{};
        L.p = p;
        L.gauge = gauge;
        L.in = (const char *)in + (1 - p) * half;
        L.aux = (const char *)in + p * half;
        L.out = (char *)out + p * half;
        L.alpha = 1.0;
        L.beta = -0.5;
        L.clov = clover_half(clover, g, rep, clover_prec(prec), false, p);
        L.clov_mode = kClovAux;
        st = launch_hop(ctx, g, rep, prec, L, s);
        if (st) return st;
    }
    return HR_OK;
}

hr_status hr_dirac_eo_clover(hr_ctx *ctx, hr_lattice lat, hr_rep rep, hr_prec prec, hr_parity out_parity, hr_op op,
                             int n_rhs, const void *gauge, const void *clover, const void *in, void *out, void *work,
                             size_t work_bytes, hr_stream stream)
{
    if (!ctx) return HR_ERR_INVALID_ARG;
    if (!clover) return set_error(ctx, HR_ERR_INVALID_ARG, "null clover field");
    if (op == HR_OP_HOP) return hr_dirac_eo(ctx, lat, 0.0, rep, prec, out_parity, op, n_rhs, gauge, in, out, work,
                                             work_bytes, stream);
    if (!valid_rep(rep) || !valid_prec(prec)) return set_error(ctx, HR_ERR_INVALID_ARG, "bad rep/prec");
    hr_status st = validate_lattice(ctx, lat, n_rhs);
    if (st) return st;
    st = check_buffers(ctx, {gauge, clover, in, out}, {}, {work});
    if (st) return st;
    if (in == out) return set_error(ctx, HR_ERR_INVALID_ARG, "in and out must not alias");
    if (op != HR_OP_SCHUR && op != HR_OP_SCHUR_DAG && op != HR_OP_NORMAL)
        return set_error(ctx, HR_ERR_INVALID_ARG, "bad op %d", (int)op);
    if (out_parity != HR_EVEN) return set_error(ctx, HR_ERR_INVALID_ARG, "Schur operators act on even sites");
    const size_t need = hr_dirac_workspace_bytes(lat, rep, prec, op, n_rhs);
    if (!work || work_bytes < need)
        return set_error(ctx, HR_ERR_WORKSPACE, "workspace of %zu bytes needed, %zu given", need, work_bytes);
    const Geom g = make_geom(lat, n_rhs);
    const size_t half = spinor_half_bytes(g, rep, prec);
    void *wo = work;
    void *we = (op == HR_OP_NORMAL) ? (char *)work + half : nullptr;
    return apply_eo_op(ctx, g, 0.0, rep, prec, op, gauge, in, out, wo, we, kFinNone, nullptr, nullptr,
                       (cudaStream_t)stream, nullptr, clover);
}

} // extern "C"

// ---------------------------------------------------------------- HMC force of the clover term
//
// Fundamental links, SW form.  For a spin-colour insertion Lam(y),
//   f = Re sum_y tr[C(y) Lam(y)] = Re sum_y (i/2) sum_{mu<nu} tr_c[F_mn(y) K_mn(y)],
// and in the chiral blocks (C+ on spins 0, 1, C- on 2, 3, as in the build), with
// P_l^b = sum_{s,t} (s_l)_st Lam[(2b+t, .), (2b+s, .)] (colour 2x2),
//   K_0l = P_l^1 - P_l^0,  K_23 = -(P_1^0 + P_1^1),  K_13 = P_2^0 + P_2^1,  K_12 = -(P_3^0 + P_3^1).
// K field: double [V][6][2][2][2] (lexicographic site, planes 01 02 03 12 13 23).
// The link derivative of f: each link lies on two plaquettes of each of the
// three planes that contain its direction, and each plaquette enters the
// leaves of its four corners; hr_clover_leaf.cuh sums the four corner
// insertions around one staple per plaquette.
//
// Two flavours of clover fermions through the even-odd pseudofermion (Mhat =
// A_ee - H_eo A_oo^-1 H_oe / 4): with X = (Mhat^+ Mhat)^-1 eta, Y = Mhat X,
// Z = A_oo^-1 H_oe X, W = A_oo^-1 H_eo^+ Y,
//   dS_pf = 1/2 dRe<a, H b> (a = (Y, W), b = (X, Z)) + c_sw df[Lam],
//   Lam = -2 X Y^+ (even), -1/2 Z W^+ (odd),
// and S_det = -2 sum_{odd} log det A adds Lam_det = -2 A^-1 (odd).

namespace {

// (s_l)_st, l = 0, 1, 2 for s_1, s_2, s_3
__device__ __forceinline__ zc pauli(int l, int s, int t)
{
    if (l == 0) return {s != t ? 1.0 : 0.0, 0.0};
    if (l == 1) return s == t ? zc{0.0, 0.0} : (s == 0 ? zc{0.0, -1.0} : zc{0.0, 1.0});
    return {s != t ? 0.0 : (s == 0 ? 1.0 : -1.0), 0.0};
}

// P[b][l][d][c] += coef * lam((2b+t, d), (2b+s, c)) summed with (s_l)_st
template <class Lam> __device__ void add_blocks(zc (&P)[2][3][2][2], double coef, Lam lam)
{
    for (int b = 0; b < 2; ++b)
        for (int l = 0; l < 3; ++l)
            for (int d = 0; d < 2; ++d)
                for (int c = 0; c < 2; ++c) {
                    zc acc = {0.0, 0.0};
                    for (int s = 0; s < 2; ++s)
                        for (int t = 0; t < 2; ++t) {
                            const zc sg = pauli(l, s, t);
                            if (sg.re == 0.0 && sg.im == 0.0) continue;
                            acc = zadd(acc, zmul(sg, lam(2 * b + t, d, 2 * b + s, c)));
                        }
                    P[b][l][d][c] = zadd(P[b][l][d][c], zscale(coef, acc));
                }
}

__device__ void store_k(double *K, long long x, const zc (&P)[2][3][2][2])
{
    for (int d = 0; d < 2; ++d)
        for (int c = 0; c < 2; ++c) {
            zc k[6];
            k[0] = zsub(P[1][0][d][c], P[0][0][d][c]);
            k[1] = zsub(P[1][1][d][c], P[0][1][d][c]);
            k[2] = zsub(P[1][2][d][c], P[0][2][d][c]);
            k[3] = zscale(-1.0, zadd(P[0][2][d][c], P[1][2][d][c])); // 12: -(P_3^0 + P_3^1)
            k[4] = zadd(P[0][1][d][c], P[1][1][d][c]);               // 13: P_2^0 + P_2^1
            k[5] = zscale(-1.0, zadd(P[0][0][d][c], P[1][0][d][c])); // 23: -(P_1^0 + P_1^1)
            for (int pl = 0; pl < 6; ++pl) {
                double *o = K + ((x * 6 + pl) * 4 + d * 2 + c) * 2;
                o[0] = k[pl].re;
                o[1] = k[pl].im;
            }
        }
}

// K from a canonical insertion Lam: complex [V][8][8], index spin * 2 + colour
__global__ void k_clover_k_from_lam(long long V, const double *lam, double *K)
{
    const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= V) return;
    const double *L = lam + x * 128;
    zc P[2][3][2][2] = {};
    add_blocks(P, 1.0, [&](int t, int d, int s, int c) {
        const int r = t * 2 + d, q = s * 2 + c;
        return zc{L[(r * 8 + q) * 2], L[(r * 8 + q) * 2 + 1]};
    });
    store_k(K, x, P);
}

struct KFieldArgs {
    Geom g;
    const void *X, *Y; // even halves (packed FP64)
    const void *Z, *W; // odd halves
    const void *ainv;  // A^-1 odd half-field (packed FP64 clover), or nullptr: no det term
    const void *afwd[2]; // exponential form: A on even / odd sites
    int exp_kind;        // 1: A = a exp(c_sw C / a), the insertion goes through exp_insertion
    double a;            // 4 + m0
    double *K;
};

// Exponential form: Lam' = int_0^1 exp((1-s) X) Lam exp(s X) ds per chiral block,
// from the eigen-decomposition of the block of A = a exp(X) (eigenvalues mu =
// a e^l): (V^+ Lam' V)_ij = (V^+ Lam V)_ij (e^l_i - e^l_j) / (l_i - l_j).
__device__ void exp_insertion_block(const zd (&Ab)[4][4], double a, zd (&L)[4][4])
{
    zd M[4][4], V[4][4];
    double mu[4], l[4];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) M[i][j] = Ab[i][j];
    jacobi_eigh<4>(M, V, mu);
    for (int i = 0; i < 4; ++i) l[i] = log(mu[i] / a);
    zd T[4][4], R[4][4];
    for (int i = 0; i < 4; ++i) // T = V^+ L V
        for (int j = 0; j < 4; ++j) {
            zc acc = {0.0, 0.0};
            for (int k = 0; k < 4; ++k)
                for (int m = 0; m < 4; ++m)
                    acc = zadd(acc, zmul(zmul(zconj(zc{V[k][i].re, V[k][i].im}), zc{L[k][m].re, L[k][m].im}),
                                         zc{V[m][j].re, V[m][j].im}));
            const double d = l[i] - l[j];
            const double phi = fabs(d) > 1e-8 ? (exp(l[i]) - exp(l[j])) / d : exp(0.5 * (l[i] + l[j]));
            T[i][j] = {phi * acc.re, phi * acc.im};
        }
    for (int i = 0; i < 4; ++i) // R = V T V^+
        for (int j = 0; j < 4; ++j) {
            zc acc = {0.0, 0.0};
            for (int k = 0; k < 4; ++k)
                for (int m = 0; m < 4; ++m)
                    acc = zadd(acc, zmul(zmul(zc{V[i][k].re, V[i][k].im}, zc{T[k][m].re, T[k][m].im}),
                                         zconj(zc{V[j][m].re, V[j][m].im})));
            R[i][j] = {acc.re, acc.im};
        }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) L[i][j] = R[i][j];
}

// the two 4 x 4 blocks of a packed FP64 clover half-field at site i
__device__ void read_blocks(const void *half, int i, zd (&M)[2][4][4])
{
    CloverReader<2, kF64, dd> rd(half, i); // double-float reals, converted exactly
    int q = 0;
    for (int b = 0; b < 2; ++b) {
        for (int k = 0; k < 4; ++k) M[b][k][k] = {dd_to_double(rd.get(q++)), 0.0};
        for (int r = 0; r < 4; ++r)
            for (int c = r + 1; c < 4; ++c) {
                const double re = dd_to_double(rd.get(q++)), im = dd_to_double(rd.get(q++));
                M[b][r][c] = {re, im};
                M[b][c][r] = {re, -im};
            }
    }
}

// K of the two-flavour clover pseudofermion (and det A_oo) insertion
__global__ void k_clover_k_from_fields(KFieldArgs A)
{
    const Geom &g = A.g;
    const long long V = 2LL * g.vh;
    const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= V) return;
    int c4[4];
    long long r = x;
    for (int k = 3; k >= 0; --k) {
        c4[k] = (int)(r % g.d[k]);
        r /= g.d[k];
    }
    const int p = (c4[0] + c4[1] + c4[2] + c4[3]) & 1;
    const int i = (int)(x >> 1);
    zc P[2][3][2][2] = {};
    cpx<double> u[4][2], v[4][2];
    load_spinor<2, kF64>(p == 0 ? A.X : A.Z, g.nblk_s, i, u);
    load_spinor<2, kF64>(p == 0 ? A.Y : A.W, g.nblk_s, i, v);
    // Lam = coef u v^+ : Lam[(t, d), (s, c)] = coef u[t][d] conj(v[s][c])
    const double coef = p == 0 ? -2.0 : -0.5;
    if (A.exp_kind) {
        zd Ab[2][4][4], Lb[2][4][4];
        read_blocks(A.afwd[p], i, Ab);
        for (int b = 0; b < 2; ++b) {
            for (int k = 0; k < 4; ++k)
                for (int m = 0; m < 4; ++m) {
                    const zc z = zmul(zc{u[2 * b + k / 2][k % 2].re, u[2 * b + k / 2][k % 2].im},
                                      zconj(zc{v[2 * b + m / 2][m % 2].re, v[2 * b + m / 2][m % 2].im}));
                    Lb[b][k][m] = {coef * z.re, coef * z.im};
                }
            exp_insertion_block(Ab[b], A.a, Lb[b]);
        }
        add_blocks(P, 1.0, [&](int t, int d, int s, int c) {
            const zd z = Lb[t >> 1][(t & 1) * 2 + d][(s & 1) * 2 + c];
            return zc{z.re, z.im};
        });
        store_k(A.K, x, P);
        return;
    }
    add_blocks(P, coef, [&](int t, int d, int s, int c) {
        return zmul(zc{u[t][d].re, u[t][d].im}, zconj(zc{v[s][c].re, v[s][c].im}));
    });
    if (p == 1 && A.ainv) {
        // Lam_det = -2 A^-1: block b (spins 2b, 2b+1) as n = 4 reals per diagonal, then the upper triangle
        // (double-float reals, converted exactly)
        CloverReader<2, kF64, dd> rd(A.ainv, i);
        zc M[2][4][4];
        int q = 0;
        for (int b = 0; b < 2; ++b) {
            for (int k = 0; k < 4; ++k) M[b][k][k] = {dd_to_double(rd.get(q++)), 0.0};
            for (int a = 0; a < 4; ++a)
                for (int c = a + 1; c < 4; ++c) {
                    const double re = dd_to_double(rd.get(q++)), im = dd_to_double(rd.get(q++));
                    M[b][a][c] = {re, im};
                    M[b][c][a] = {re, -im};
                }
        }
        add_blocks(P, -2.0, [&](int t, int d, int s, int c) {
            const int b = t >> 1; // same block as s (diagonal blocks only are read)
            return M[b][(t & 1) * 2 + d][(s & 1) * 2 + c];
        });
    }
    store_k(A.K, x, P);
}

// F[rho][z][a] += scale * d/dw_a Re sum_y tr[C Lam], one thread per link (rho, z):
// the two plaquettes of each of the three planes that hold rho, each with its
// four corner insertions around one staple (hr_clover_leaf.cuh)
__global__ void __launch_bounds__(128) k_clover_leaf_force(Geom g, const double *can, const double *K, double scale,
                                                           double *F)
{
    const long long V = 2LL * g.vh;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 4 * V) return;
    const int rho = (int)(t / V);
    const long long z = t - (long long)rho * V;
    int x[4];
    long long r = z;
    for (int k = 3; k >= 0; --k) {
        x[k] = (int)(r % g.d[k]);
        r /= g.d[k];
    }
    LeafLattice L;
    for (int k = 0; k < 4; ++k) L.d[k] = g.d[k];
    double out[3];
    leaf_force_link(L, can, K, rho, x, out);
    double *o = F + ((long long)rho * V + z) * 3;
    for (int a = 0; a < 3; ++a) o[a] += scale * out[a];
}

// block sums of sum_{odd sites} log det A (both blocks, Cholesky), one partial per block
template <int NC> __global__ void __launch_bounds__(128) k_clover_logdet(Geom g, const void *half, double *partial,
                                                                         unsigned *bad)
{
    constexpr int N = 2 * NC;
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.vh; i += gridDim.x * blockDim.x) {
        CloverReader<NC, kF64, dd> rd(half, i); // double-float reals, converted exactly
        int q = 0;
        for (int b = 0; b < 2; ++b) {
            zc M[N][N];
            for (int k = 0; k < N; ++k) M[k][k] = {dd_to_double(rd.get(q++)), 0.0};
            for (int a = 0; a < N; ++a)
                for (int c = a + 1; c < N; ++c) {
                    const double re = dd_to_double(rd.get(q++)), im = dd_to_double(rd.get(q++));
                    M[a][c] = {re, im};
                    M[c][a] = {re, -im};
                }
            // Cholesky M = L L^+ in place (lower triangle); log det = 2 sum log L_kk
            for (int k = 0; k < N; ++k) {
                double dkk = M[k][k].re;
                for (int j = 0; j < k; ++j) dkk -= M[k][j].re * M[k][j].re + M[k][j].im * M[k][j].im;
                if (!(dkk > 0.0)) {
                    atomicExch(bad, 1u);
                    dkk = 1.0;
                }
                const double lkk = sqrt(dkk);
                acc += 2.0 * log(lkk);
                for (int a = k + 1; a < N; ++a) {
                    zc s = M[a][k];
                    for (int j = 0; j < k; ++j) s = zsub(s, zmul(M[a][j], zconj(M[k][j])));
                    M[a][k] = zscale(1.0 / lkk, s);
                }
            }
        }
    }
    __shared__ double red[128];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

constexpr int kLogdetBlocks = 256;

size_t k_field_bytes(const Geom &g) { return ((size_t)2 * g.vh * 48 * sizeof(double) + 255) & ~(size_t)255; }

hr_status leaf_force(hr_ctx *ctx, const Geom &g, const double *can, const double *K, double scale, double *F,
                     cudaStream_t s)
{
    const long long n = 8LL * g.vh;
    k_clover_leaf_force<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(g, can, K, scale, F);
    return check_launch(ctx, "clover force");
}

} // namespace

extern "C" {

size_t hr_clover_force_workspace_bytes(hr_lattice lat)
{
    if (hr_gauge_packed_bytes(lat, HR_FUND, HR_F64) == 0) return 0;
    const Geom g = make_geom(lat, 1);
    const size_t half = spinor_half_bytes(g, HR_FUND, kF64);
    return k_field_bytes(g) + 5 * half;
}

hr_status hr_clover_insertion_force(hr_ctx *ctx, hr_lattice lat, double c_sw, const double *gauge, const double *lam,
                                    double coeff, double *force, void *work, size_t work_bytes, hr_stream stream)
{
    if (!ctx) return HR_ERR_INVALID_ARG;
    hr_status st = validate_lattice(ctx, lat, 1);
    if (st) return st;
    st = check_buffers(ctx, {work}, {gauge, lam, force});
    if (st) return st;
    if (!std::isfinite(c_sw) || !std::isfinite(coeff)) return set_error(ctx, HR_ERR_INVALID_ARG, "c_sw, coeff finite");
    const Geom g = make_geom(lat, 1);
    if (work_bytes < k_field_bytes(g))
        return set_error(ctx, HR_ERR_WORKSPACE, "workspace of %zu bytes needed, %zu given", k_field_bytes(g), work_bytes);
    cudaStream_t s = (cudaStream_t)stream;
    const long long V = 2LL * g.vh;
    k_clover_k_from_lam<<<(unsigned)((V + 127) / 128), 128, 0, s>>>(V, lam, (double *)work);
    st = check_launch(ctx, "clover insertion");
    if (!st) st = leaf_force(ctx, g, gauge, (const double *)work, coeff * c_sw, force, s);
    return st;
}

hr_status hr_clover_fermion_force(hr_ctx *ctx, hr_lattice lat, hr_clover_kind kind, double m0, double c_sw,
                                  const double *gauge, const void *gauge_packed, const void *clover, const void *X,
                                  const void *Y, int with_det, double coeff, double *force, void *work,
                                  size_t work_bytes, hr_stream stream)
{
    if (ctx && kind != HR_CLOVER_SW && kind != HR_CLOVER_EXP)
        return set_error(ctx, HR_ERR_INVALID_ARG, "bad clover kind");
    if (!ctx) return HR_ERR_INVALID_ARG;
    hr_status st = validate_lattice(ctx, lat, 1);
    if (st) return st;
    st = check_buffers(ctx, {gauge_packed, clover, X, work}, {gauge, force}, {Y});
    if (st) return st;
    if (!(4.0 + m0 != 0.0) || !std::isfinite(c_sw) || !std::isfinite(coeff))
        return set_error(ctx, HR_ERR_INVALID_ARG, "4 + m0 nonzero, c_sw and coeff finite");
    const size_t need = hr_clover_force_workspace_bytes(lat);
    if (work_bytes < need) return set_error(ctx, HR_ERR_WORKSPACE, "workspace of %zu bytes needed, %zu given", need, work_bytes);
    const Geom g = make_geom(lat, 1);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t half = spinor_half_bytes(g, HR_FUND, kF64);
    char *w = (char *)work;
    double *K = (double *)w;
    char *a = w + k_field_bytes(g);  // full field (Y | W)
    char *b = a + 2 * half;          // full field (X | Z)
    char *t_odd = b + 2 * half;
    const void *ainv_odd = clover_half(clover, g, HR_FUND, kF64, true, 1);
    // Y = Mhat X, or the given Y
    if (Y) {
        cudaError_t ce = cudaMemcpyAsync(a, Y, half, cudaMemcpyDeviceToDevice, s);
        if (ce != cudaSuccess) return set_error(ctx, HR_ERR_CUDA, "copy: %s", cudaGetErrorString(ce));
    } else {
        st = apply_eo_op(ctx, g, m0, HR_FUND, kF64, HR_OP_SCHUR, gauge_packed, X, a, t_odd, nullptr, kFinNone,
                         nullptr, nullptr, s, nullptr, clover);
        if (st) return st;
    }
    // Z = A_oo^-1 H_oe X,  W = A_oo^-1 g5 H_oe g5 Y  (A commutes with g5)
    for (int k = 0; k < 2; ++k) {
        HopLaunch L{};
        L.p = 1;
        L.gauge = gauge_packed;
        L.in = k == 0 ? X : (const void *)a;
        L.out = k == 0 ? b + half : a + half;
        L.beta = 1.0;
        L.g5_in = L.g5_out = k;
        L.clov = ainv_odd;
        L.clov_mode = kClovOut;
        st = launch_hop(ctx, g, HR_FUND, kF64, L, s);
        if (st) return st;
    }
    cudaError_t e = cudaMemcpyAsync(b, X, half, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return set_error(ctx, HR_ERR_CUDA, "copy: %s", cudaGetErrorString(e));
    // the hops: 1/2 dRe<a, H b>
    st = hr_force(ctx, lat, gauge_packed, a, b, 0.5 * coeff, force, stream);
    if (st) return st;
    // the site term: c_sw df[Lam]
    KFieldArgs A;
    A.g = g;
    A.X = b;
    A.Y = a;
    A.Z = b + half;
    A.W = a + half;
    // the exponential form's det A_oo is a constant (C is traceless): no det force
    A.ainv = (with_det && kind == HR_CLOVER_SW) ? ainv_odd : nullptr;
    A.afwd[0] = clover_half(clover, g, HR_FUND, kF64, false, 0);
    A.afwd[1] = clover_half(clover, g, HR_FUND, kF64, false, 1);
    A.exp_kind = kind == HR_CLOVER_EXP;
    A.a = 4.0 + m0;
    A.K = K;
    const long long V = 2LL * g.vh;
    k_clover_k_from_fields<<<(unsigned)((V + 127) / 128), 128, 0, s>>>(A);
    st = check_launch(ctx, "clover insertion");
    if (!st) st = leaf_force(ctx, g, gauge, K, coeff * c_sw, force, s);
    return st;
}

hr_status hr_clover_logdet(hr_ctx *ctx, hr_lattice lat, hr_rep rep, const void *clover, hr_parity parity,
                           double *logdet, hr_stream stream)
{
    if (!ctx) return HR_ERR_INVALID_ARG;
    if (!logdet) return set_error(ctx, HR_ERR_INVALID_ARG, "null result pointer");
    if (rep != HR_FUND && rep != HR_ADJ) return set_error(ctx, HR_ERR_INVALID_ARG, "HR_FUND or HR_ADJ");
    if (parity != HR_EVEN && parity != HR_ODD) return set_error(ctx, HR_ERR_INVALID_ARG, "bad parity");
    hr_status st = validate_lattice(ctx, lat, 1);
    if (st) return st;
    st = check_buffers(ctx, {clover});
    if (st) return st;
    const Geom g = make_geom(lat, 1);
    cudaStream_t s = (cudaStream_t)stream;
    const void *half = clover_half(clover, g, rep, kF64, false, parity);
    unsigned *bad = ctx->d_counters + C_STATUS;
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return set_error(ctx, HR_ERR_CUDA, "status reset: %s", cudaGetErrorString(e));
    if (rep == HR_FUND) k_clover_logdet<2><<<kLogdetBlocks, 128, 0, s>>>(g, half, ctx->d_partials, bad);
    else k_clover_logdet<3><<<kLogdetBlocks, 128, 0, s>>>(g, half, ctx->d_partials, bad);
    st = check_launch(ctx, "clover log det");
    if (st) return st;
    double h[kLogdetBlocks];
    unsigned hb = 0;
    e = cudaMemcpyAsync(h, ctx->d_partials, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hb, bad, sizeof hb, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_error(ctx, HR_ERR_CUDA, "log det readback: %s", cudaGetErrorString(e));
    if (hb) return set_error(ctx, HR_ERR_NUMERIC, "a clover block is not positive definite");
    double acc = 0.0;
    for (int k = 0; k < kLogdetBlocks; ++k) acc += h[k];
    *logdet = acc;
    return HR_OK;
}

} // extern "C"
