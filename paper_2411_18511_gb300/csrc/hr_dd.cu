// hr_dd.cu -- the hop on a lattice split along time into slabs, one per GPU
// (the paper's multi-GPU organisation, Sec. 2.1.1: inner sites computed while
// the boundary data travels, then the boundary sites).
//
// Each rank holds a slab of T_loc = T / n time slices (T_loc even, so local
// and global parities agree) as an ordinary local lattice.  A hop of the
// local lattice with the library's tuned kernels wraps time inside the slab:
// every term is right except the time hops of the two face slices, which
// must reach the neighbouring slabs.  Those are exchanged as half spinors:
//
//   to_lower (for the rank below):  P-_0 psi(x)             on the slice t = 0
//   to_upper (for the rank above):  U_0(x)^+ P+_0 psi(x)    on the slice t = T_loc - 1
//
// with P-+_0 = (1 -+ g_0) projected to two spins (the forward term of the
// receiver needs its own link U_0 on top of P- psi; the backward term needs
// the sender's link, so the sender applies it).  After the exchange the
// boundary kernel replaces, on the face slices of the output parity, the
// wrapped time term by the received one:
//
//   top slice:     out += beta (1 - g_0) U_0(x) [from_upper - P-_0 psi(x + 0, wrapped)]
//   bottom slice:  out += beta (1 + g_0) [from_lower - U_0(x - 0, wrapped)^+ P+_0 psi(x - 0, wrapped)]
//
// in the hop's arithmetic (double-float for HR_F64).  A face slice of a
// parity has V3/2 sites (V3 = L1 L2 L3), numbered by their even-odd index
// within the slice; the slab below's top slice and the slab above's bottom
// slice pair up site by site.  Face buffers: 4 NC reals per face site
// (the two spins of NC complex colours), real-major ([real][site]), FP64 as
// (hi, lo) float pairs, FP32 / FP16 as floats.
#include <cmath>

#include "hr_hop_fam.h"

using namespace hr;

namespace {

// one face real, in the precision of the face
template <int PREC> struct FaceT { using T = float; using S = float; };
template <> struct FaceT<kF64> { using T = dd; using S = float2; };

template <int PREC>
__device__ __forceinline__ void face_store(void *face, int nf, int k, int f, typename FaceT<PREC>::T v)
{
    if constexpr (PREC == kF64) ((float2 *)face)[(size_t)k * nf + f] = make_float2(v.h, v.l);
    else ((float *)face)[(size_t)k * nf + f] = v;
}
template <int PREC>
__device__ __forceinline__ typename FaceT<PREC>::T face_load(const void *face, int nf, int k, int f)
{
    if constexpr (PREC == kF64) {
        const float2 w = ((const float2 *)face)[(size_t)k * nf + f];
        return dd(w.x, w.y);
    } else {
        return ((const float *)face)[(size_t)k * nf + f];
    }
}

// colour link of (parity, mu = 0, site) in the arithmetic type
template <int REP, int PREC, class T, class M>
__device__ __forceinline__ void time_link(const void *gauge, int nblk_g, int par, int i, M &link)
{
    if constexpr (REP == kRepFund) {
        load_quat<PREC>(gauge, nblk_g, par, 0, i, link);
    } else if constexpr (REP == kRepAdj) {
        T q[4];
        load_quat<PREC>(gauge, nblk_g, par, 0, i, q);
        quat_to_adj(q, link);
    } else {
        load_mat<PREC>(gauge, nblk_g, par, 0, i, link);
    }
}

template <int REP, class T> struct LinkT;
template <class T> struct LinkT<kRepFund, T> { using M = T[4]; };
template <class T> struct LinkT<kRepAdj, T> { using M = T[3][3]; };
template <class T> struct LinkT<kRepAdjMat, T> { using M = T[3][3]; };

template <bool DAG, int REP, class T, int NC, class M>
__device__ __forceinline__ void colour_mul(const M &link, const cpx<T> (&h)[NC], cpx<T> (&r)[NC])
{
    if constexpr (REP == kRepFund) su2_mul<DAG>(link, h, r);
    else so3_mul<DAG>(link, h, r);
}

// Faces of the input field `in` (parity q = par of the local lattice); one
// thread per face site f.
template <int REP, int PREC>
__global__ void k_dd_pack(Geom g, int par, const void *gauge, const void *in, void *to_lower, void *to_upper, int nf)
{
    using T = typename PrecTraits<PREC>::T;
    constexpr int NC = RepTraits<REP>::NC;
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    cpx<T> s[4][NC], h[2][NC];
    // bottom slice t = 0: P-_0 psi
    load_spinor<NC, PREC>(in, g.nblk_s, f, s);
    spin_project<0, true>(s, h);
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            face_store<PREC>(to_lower, nf, 2 * (NC * t + c), f, h[t][c].re);
            face_store<PREC>(to_lower, nf, 2 * (NC * t + c) + 1, f, h[t][c].im);
        }
    // top slice t = T_loc - 1: U_0(x)^+ P+_0 psi
    const int it = (g.d[0] - 1) * nf + f;
    load_spinor<NC, PREC>(in, g.nblk_s, it, s);
    spin_project<0, false>(s, h);
    typename LinkT<REP, T>::M link;
    time_link<REP, PREC, T>(gauge, g.nblk_g, par, it, link);
    cpx<T> r[2][NC];
    colour_mul<true, REP>(link, h[0], r[0]);
    colour_mul<true, REP>(link, h[1], r[1]);
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            face_store<PREC>(to_upper, nf, 2 * (NC * t + c), f, r[t][c].re);
            face_store<PREC>(to_upper, nf, 2 * (NC * t + c) + 1, f, r[t][c].im);
        }
}

// Replace the wrapped time terms of the face sites of output parity p by the
// received ones (see the file comment).  `in` holds the input parity 1 - p.
template <int REP, int PREC>
__global__ void k_dd_boundary(Geom g, int p, const void *gauge, const void *in, const void *from_lower,
                              const void *from_upper, void *out, coef2 beta, int nf)
{
    using T = typename PrecTraits<PREC>::T;
    constexpr int NC = RepTraits<REP>::NC;
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    const T be = Real<T>::from_coef(beta);
    const int top = (g.d[0] - 1) * nf + f;
    cpx<T> s[4][NC], h[2][NC], r[2][NC], acc[4][NC], o[4][NC];
    // top slice of parity p: forward time term, link U_0(x) at the output site
    {
        load_spinor<NC, PREC>(in, g.nblk_s, f, s); // the wrapped neighbour: t = 0 of this slab
        spin_project<0, true>(s, h);
#pragma unroll
        for (int t = 0; t < 2; ++t)
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const T re = face_load<PREC>(from_upper, nf, 2 * (NC * t + c), f);
                const T im = face_load<PREC>(from_upper, nf, 2 * (NC * t + c) + 1, f);
                h[t][c] = {re - h[t][c].re, im - h[t][c].im};
            }
        typename LinkT<REP, T>::M link;
        time_link<REP, PREC, T>(gauge, g.nblk_g, p, top, link);
        colour_mul<false, REP>(link, h[0], r[0]);
        colour_mul<false, REP>(link, h[1], r[1]);
        spin_accumulate<0, true, T, NC, true>(acc, r);
        load_spinor<NC, PREC>(out, g.nblk_s, top, o);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < NC; ++c)
                o[a][c] = {o[a][c].re + be * acc[a][c].re, o[a][c].im + be * acc[a][c].im};
        store_spinor<NC, PREC>(out, g.nblk_s, top, o);
    }
    // bottom slice of parity p: backward time term from the slab below
    {
        load_spinor<NC, PREC>(in, g.nblk_s, top, s); // the wrapped neighbour: t = T_loc - 1
        spin_project<0, false>(s, h);
        typename LinkT<REP, T>::M link;
        time_link<REP, PREC, T>(gauge, g.nblk_g, 1 - p, top, link);
        colour_mul<true, REP>(link, h[0], r[0]);
        colour_mul<true, REP>(link, h[1], r[1]);
#pragma unroll
        for (int t = 0; t < 2; ++t)
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const T re = face_load<PREC>(from_lower, nf, 2 * (NC * t + c), f);
                const T im = face_load<PREC>(from_lower, nf, 2 * (NC * t + c) + 1, f);
                r[t][c] = {re - r[t][c].re, im - r[t][c].im};
            }
        spin_accumulate<0, false, T, NC, true>(acc, r);
        load_spinor<NC, PREC>(out, g.nblk_s, f, o);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < NC; ++c)
                o[a][c] = {o[a][c].re + be * acc[a][c].re, o[a][c].im + be * acc[a][c].im};
        store_spinor<NC, PREC>(out, g.nblk_s, f, o);
    }
}

template <int REP, int PREC> struct DdLaunch {
    static bool run(const Geom &g, bool pack, int par, const void *gauge, const void *in, const void *fa,
                    const void *fb, void *out, double beta, cudaStream_t s)
    {
        const int nf = g.d[1] * g.d[2] * g.d[3] / 2;
        const int bs = 128, grid = (nf + bs - 1) / bs;
        if (pack) k_dd_pack<REP, PREC><<<grid, bs, 0, s>>>(g, par, gauge, in, (void *)fa, (void *)fb, nf);
        else k_dd_boundary<REP, PREC><<<grid, bs, 0, s>>>(g, par, gauge, in, fa, fb, out, make_coef(beta), nf);
        return true;
    }
};

hr_status dd_check(hr_ctx *ctx, const hr_lattice &local, int rep, int prec, int parity)
{
    if (!valid_rep(rep) || !valid_prec(prec)) return set_error(ctx, HR_ERR_INVALID_ARG, "bad rep/prec");
    hr_status st = validate_lattice(ctx, local, 1);
    if (st) return st;
    if (parity != HR_EVEN && parity != HR_ODD) return set_error(ctx, HR_ERR_INVALID_ARG, "bad parity");
    if (local.theta[0] != 0.0)
        return set_error(ctx, HR_ERR_UNSUPPORTED, "a twist in the split (time) direction is not supported");
    return HR_OK;
}

} // namespace

extern "C" {

size_t hr_dd_face_bytes(hr_lattice local, hr_rep rep, hr_prec prec)
{
    if (!valid_rep(rep) || !valid_prec(prec)) return 0;
    if (hr_spinor_packed_bytes(local, rep, prec, HR_EVEN, 1) == 0) return 0;
    const size_t nf = (size_t)local.dims[1] * local.dims[2] * local.dims[3] / 2;
    const size_t b = nf * 4 * rep_nc(rep) * (prec == HR_F64 ? 8 : 4);
    return (b + 255) & ~(size_t)255;
}

hr_status hr_dd_pack_faces(hr_ctx *ctx, hr_lattice local, hr_rep rep, hr_prec prec, hr_parity in_parity,
                           const void *gauge, const void *in, void *to_lower, void *to_upper, hr_stream stream)
{
    if (!ctx) return HR_ERR_INVALID_ARG;
    hr_status st = dd_check(ctx, local, rep, prec, in_parity);
    if (st) return st;
    st = check_buffers(ctx, {gauge, in, to_lower, to_upper});
    if (st) return st;
    if (to_lower == to_upper) return set_error(ctx, HR_ERR_INVALID_ARG, "the two faces must not alias");
    const Geom g = make_geom(local, 1);
    for_config<DdLaunch>(rep, prec, g, true, (int)in_parity, gauge, in, to_lower, to_upper, nullptr, 0.0,
                         (cudaStream_t)stream);
    return check_launch(ctx, "face pack");
}

hr_status hr_dd_hop_boundary(hr_ctx *ctx, hr_lattice local, hr_rep rep, hr_prec prec, hr_parity out_parity,
                             const void *gauge, const void *in, const void *from_lower, const void *from_upper,
                             void *out, hr_stream stream)
{
    if (!ctx) return HR_ERR_INVALID_ARG;
    hr_status st = dd_check(ctx, local, rep, prec, out_parity);
    if (st) return st;
    st = check_buffers(ctx, {gauge, in, from_lower, from_upper, out});
    if (st) return st;
    if (in == out) return set_error(ctx, HR_ERR_INVALID_ARG, "in and out must not alias");
    const Geom g = make_geom(local, 1);
    // the operator of HR_OP_HOP: D_{p,1-p} = -1/2 H
    for_config<DdLaunch>(rep, prec, g, false, (int)out_parity, gauge, in, from_lower, from_upper, out, -0.5,
                         (cudaStream_t)stream);
    return check_launch(ctx, "face boundary");
}

} // extern "C"
