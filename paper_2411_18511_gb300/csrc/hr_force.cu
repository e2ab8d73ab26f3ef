// hr_force.cu -- link derivatives of f = Re<a, H b> for fundamental SU(2) links:
// the su(2) fermion force of the HMC (arXiv:2411.18511 Sec. 2.1 and Sec. 2.2 name
// the HMC as the consumer of the even-odd operator) and the gradient with
// respect to the four quaternion components (used by the autograd wrappers).
//
// The two terms of H that contain U_mu(x) are
//   a(x)^+ (1-g_mu) U b(x+mu)  and  a(x+mu)^+ (1+g_mu) U^+ b(x).
// With the spin-traced colour outer products
//   M1 = sum_s b(x+mu)_s [((1-g_mu) a(x))_s]^+,   M2 = sum_s b(x)_s [((1+g_mu) a(x+mu))_s]^+
// their variation is Re tr[dU M1] + Re tr[dU^+ M2], so
//   quaternion gradient  G_k = Re tr[E_k M1] + Re tr[E_k^+ M2]  (E_0 = 1, E_k = i s_k)
//   su(2) force          F_a = Re tr[(i s_a/2)(U M1 - M2 U^+)]   for U -> exp(i w.s/2) U.
// One thread per site (both parities in one launch); it writes all four
// directions of its own links, so no two threads touch the same output.
// Boundaries: the two terms that contain a link on the boundary slice both
// cross the boundary.  An antiperiodic sign multiplies both (the packed links
// carry it; the quaternion gradient, which takes no gauge field, applies it);
// a twist e^{i theta} multiplies the forward hop's term and e^{-i theta} the
// backward hop's, i.e. M1 -> e^{i theta} M1 and M2 -> e^{-i theta} M2.
#include <cmath>

#include "hr_host.h"

using namespace hr;

namespace {

struct ForceArgs {
    Geom g;
    const void *gauge;
    const void *a[2]; // even, odd halves
    const void *b[2];
    double beta;
    double *out;
    int mode; // 0: su(2) force [4][V][3], 1: quaternion gradient [4][V][4]
    double tc[4], ts[4]; // e^{i theta_mu} of twisted directions (1, 0 otherwise)
};

struct c2 {
    double re, im;
};
__device__ __forceinline__ c2 cmul(c2 a, c2 b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ c2 cmulc(c2 a, c2 b) { return {a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im}; } // a conj(b)
__device__ __forceinline__ c2 cplus(c2 a, c2 b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ c2 cminus(c2 a, c2 b) { return {a.re - b.re, a.im - b.im}; }

// sg: -1 for a link on the boundary slice of an antiperiodic direction.  The
// force reads the packed links, which carry that sign already; the quaternion
// gradient takes no gauge field and applies it here.  edge: the link lies on
// the boundary slice (x_mu = L_mu - 1), where a twist applies.
template <int MU>
__device__ __forceinline__ void link_terms(const ForceArgs &A, int p, int i, int ifw, long long lex, double sg,
                                           bool edge)
{
    const Geom &g = A.g;
    cpx<double> ax[4][2], axf[4][2], bx[4][2], bxf[4][2];
    load_spinor<2, kF64>(A.a[p], g.nblk_s, i, ax);
    load_spinor<2, kF64>(A.a[1 - p], g.nblk_s, ifw, axf);
    load_spinor<2, kF64>(A.b[p], g.nblk_s, i, bx);
    load_spinor<2, kF64>(A.b[1 - p], g.nblk_s, ifw, bxf);
    // full (1 - g) a(x) and (1 + g) a(x+mu) from their half spinors
    cpx<double> h[2][2], pa[4][2], pb[4][2];
    for (int s = 0; s < 4; ++s)
        for (int c = 0; c < 2; ++c) pa[s][c] = pb[s][c] = {0.0, 0.0};
    spin_project<MU, true>(ax, h);
    spin_accumulate<MU, true>(pa, h);
    spin_project<MU, false>(axf, h);
    spin_accumulate<MU, false>(pb, h);
    c2 M1[2][2], M2[2][2];
    for (int c = 0; c < 2; ++c)
        for (int d = 0; d < 2; ++d) {
            c2 s1 = {0, 0}, s2 = {0, 0};
            for (int s = 0; s < 4; ++s) {
                s1 = cplus(s1, cmulc({bxf[s][c].re, bxf[s][c].im}, {pa[s][d].re, pa[s][d].im}));
                s2 = cplus(s2, cmulc({bx[s][c].re, bx[s][c].im}, {pb[s][d].re, pb[s][d].im}));
            }
            M1[c][d] = s1;
            M2[c][d] = s2;
        }
    if (edge && A.g.twisted) {
        const c2 f = {A.tc[MU], A.ts[MU]}, fb = {A.tc[MU], -A.ts[MU]};
        for (int c = 0; c < 2; ++c)
            for (int d = 0; d < 2; ++d) {
                M1[c][d] = cmul(f, M1[c][d]);
                M2[c][d] = cmul(fb, M2[c][d]);
            }
    }
    const long long V = 2LL * g.vh;
    if (A.mode == 1) {
        // tr(s_1 M) = M10 + M01, tr(s_2 M) = i (M01 - M10), tr(s_3 M) = M00 - M11
        c2 t1[3], t2[3];
        t1[0] = cplus(M1[1][0], M1[0][1]);
        t1[1] = {-(M1[0][1].im - M1[1][0].im), M1[0][1].re - M1[1][0].re};
        t1[2] = cminus(M1[0][0], M1[1][1]);
        t2[0] = cplus(M2[1][0], M2[0][1]);
        t2[1] = {-(M2[0][1].im - M2[1][0].im), M2[0][1].re - M2[1][0].re};
        t2[2] = cminus(M2[0][0], M2[1][1]);
        double G[4];
        G[0] = M1[0][0].re + M1[1][1].re + M2[0][0].re + M2[1][1].re;
        for (int k = 0; k < 3; ++k) G[k + 1] = -t1[k].im + t2[k].im;
        double *o = A.out + ((long long)MU * V + lex) * 4;
        for (int k = 0; k < 4; ++k) o[k] += sg * A.beta * G[k];
    } else {
        double q[4];
        load_quat<kF64>(A.gauge, g.nblk_g, p, MU, i, q);
        // U = [[q0 + i q3, q2 + i q1], [-q2 + i q1, q0 - i q3]]
        c2 U[2][2] = {{{q[0], q[3]}, {q[2], q[1]}}, {{-q[2], q[1]}, {q[0], -q[3]}}};
        c2 Q[2][2];
        for (int c = 0; c < 2; ++c)
            for (int d = 0; d < 2; ++d) {
                c2 um = cplus(cmul(U[c][0], M1[0][d]), cmul(U[c][1], M1[1][d]));       // (U M1)_cd
                c2 mu = cplus(cmulc(M2[c][0], U[d][0]), cmulc(M2[c][1], U[d][1]));     // (M2 U^+)_cd
                Q[c][d] = cminus(um, mu);
            }
        // F_a = Re[(i/2) tr(s_a Q)] = -1/2 Im tr(s_a Q)
        double F[3];
        F[0] = -0.5 * (Q[0][1].im + Q[1][0].im);
        F[1] = -0.5 * (Q[0][1].re - Q[1][0].re);
        F[2] = -0.5 * (Q[0][0].im - Q[1][1].im);
        double *o = A.out + ((long long)MU * V + lex) * 3;
        for (int k = 0; k < 3; ++k) o[k] += A.beta * F[k];
    }
}

__global__ void k_link_deriv(ForceArgs A)
{
    const Geom &g = A.g;
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * g.vh) return;
    int p = t >= g.vh ? 1 : 0;
    int i = t - p * g.vh;
    SiteNb nb;
    site_neighbours(g, i, p, nb);
    long long lex = eo_to_lex(g, i, p);
    // coordinates of the site: boundary slices of the antiperiodic directions
    int x[4];
    long long r = lex;
    for (int k = 3; k >= 0; --k) {
        x[k] = (int)(r % g.d[k]);
        r /= g.d[k];
    }
    auto sg = [&](int mu) { return (A.mode == 1 && ((g.bc >> mu) & 1) && x[mu] == g.d[mu] - 1) ? -1.0 : 1.0; };
    link_terms<0>(A, p, i, nb.fwd[0], lex, sg(0), x[0] == g.d[0] - 1);
    link_terms<1>(A, p, i, nb.fwd[1], lex, sg(1), x[1] == g.d[1] - 1);
    link_terms<2>(A, p, i, nb.fwd[2], lex, sg(2), x[2] == g.d[2] - 1);
    link_terms<3>(A, p, i, nb.fwd[3], lex, sg(3), x[3] == g.d[3] - 1);
}

hr_status launch(hr_ctx *ctx, hr_lattice lat, const void *gauge, const void *af, const void *bf, double beta,
                 double *out, int mode, hr_stream stream)
{
    if (!ctx) return HR_ERR_INVALID_ARG;
    hr_status st = validate_lattice(ctx, lat, 1);
    if (st) return st;
    if (mode == 0 && !gauge) return set_error(ctx, HR_ERR_INVALID_ARG, "null pointer");
    st = check_buffers(ctx, {af, bf}, {out}, {gauge});
    if (st) return st;
    ForceArgs A;
    A.g = make_geom(lat, 1);
    size_t half = spinor_half_bytes(A.g, HR_FUND, kF64);
    A.gauge = gauge;
    A.a[0] = af;
    A.a[1] = (const char *)af + half;
    A.b[0] = bf;
    A.b[1] = (const char *)bf + half;
    A.beta = beta;
    A.out = out;
    A.mode = mode;
    for (int k = 0; k < 4; ++k) {
        A.tc[k] = std::cos(lat.theta[k]);
        A.ts[k] = std::sin(lat.theta[k]);
    }
    int bs = 128;
    int grid = (int)((2LL * A.g.vh + bs - 1) / bs);
    k_link_deriv<<<grid, bs, 0, (cudaStream_t)stream>>>(A);
    return check_launch(ctx, mode ? "link grad" : "force");
}

// Link derivative of B(X, L) = Re<L, Mhat^+ Mhat X> at fixed even fields X, L
// (Sec. 2.1: the even-odd operator in the HMC).  With Mhat = (4+m0) - c H_eo H_oe,
// c = 1 / (4 (4+m0)), and H_eo^+ = g5 H_oe g5,
//   dB = Re<Mhat L, dMhat X> + Re<Mhat X, dMhat L>,
//   Re<Y, dMhat Z> = -c dRe<(Y, H_eo^+ Y), H (Z, H_oe Z)>,
// so each of the two terms is one application of the hop derivative (mode 0:
// su(2) force, 1: quaternion gradient) to full fields a = (Mhat Y, H_eo^+ Mhat Y)
// and b = (Z, H_oe Z) assembled in the work buffer: L = X needs one (doubled).
struct FermionWork {
    char *a, *b, *t; // two full fields and an odd temporary
    static size_t bytes(const Geom &g)
    {
        const size_t half = spinor_half_bytes(g, HR_FUND, kF64);
        return 5 * half;
    }
};

hr_status fermion_deriv(hr_ctx *ctx, hr_lattice lat, double m0, hr_rep rep, const void *gauge, const void *X,
                        const void *L, double coeff, double *out, int mode, void *work, size_t work_bytes,
                        hr_stream stream)
{
    if (!ctx) return HR_ERR_INVALID_ARG;
    if (!valid_rep(rep)) return set_error(ctx, HR_ERR_INVALID_ARG, "bad rep");
    if (rep != HR_FUND)
        return set_error(ctx, HR_ERR_UNSUPPORTED, "the fermion force is implemented for fundamental links only");
    hr_status st = validate_lattice(ctx, lat, 1);
    if (st) return st;
    st = check_buffers(ctx, {gauge, X, work}, {out}, {L});
    if (st) return st;
    if (!(4.0 + m0 != 0.0) || !std::isfinite(m0)) return set_error(ctx, HR_ERR_INVALID_ARG, "4 + m0 must be nonzero");
    if (!std::isfinite(coeff)) return set_error(ctx, HR_ERR_INVALID_ARG, "coeff is not finite");
    const Geom g = make_geom(lat, 1);
    const size_t half = spinor_half_bytes(g, HR_FUND, kF64);
    const size_t need = FermionWork::bytes(g);
    if (work_bytes < need)
        return set_error(ctx, HR_ERR_WORKSPACE, "workspace of %zu bytes needed, %zu given", need, work_bytes);
    cudaStream_t s = (cudaStream_t)stream;
    FermionWork w{(char *)work, (char *)work + 2 * half, (char *)work + 4 * half};
    const double c = 1.0 / (4.0 * (4.0 + m0));
    // dst_odd = [g5] H_oe [g5] src_even
    auto hop_oe = [&](const void *src, void *dst, int g5) {
        HopLaunch H{};
        H.p = 1;
        H.gauge = gauge;
        H.in = src;
        H.out = dst;
        H.beta = 1.0;
        H.g5_in = g5;
        H.g5_out = g5;
        return launch_hop(ctx, g, HR_FUND, kF64, H, s);
    };
    // out += coeff * (-c) * k * dRe<(Mhat Y, H_eo^+ Mhat Y), H (Z, H_oe Z)>
    auto term = [&](const void *Y, const void *Z, double k) {
        hr_status t = apply_eo_op(ctx, g, m0, HR_FUND, kF64, HR_OP_SCHUR, gauge, Y, w.a, w.t, nullptr, kFinNone,
                                  nullptr, nullptr, s);
        if (!t) t = hop_oe(w.a, w.a + half, 1);
        if (!t) {
            cudaError_t e = cudaMemcpyAsync(w.b, Z, half, cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) t = set_error(ctx, HR_ERR_CUDA, "copy: %s", cudaGetErrorString(e));
        }
        if (!t) t = hop_oe(Z, w.b + half, 0);
        if (!t) t = launch(ctx, lat, gauge, w.a, w.b, -c * k * coeff, out, mode, stream);
        return t;
    };
    if (!L || L == X) return term(X, X, 2.0);
    st = term(L, X, 1.0);
    if (!st) st = term(X, L, 1.0);
    return st;
}

} // namespace

extern "C" {

size_t hr_fermion_force_workspace_bytes(hr_lattice lat)
{
    return 5 * hr_spinor_packed_bytes(lat, HR_FUND, HR_F64, HR_EVEN, 1);
}

hr_status hr_fermion_force(hr_ctx *ctx, hr_lattice lat, double m0, hr_rep rep, const void *gauge, const void *X,
                           const void *L, double coeff, double *force, void *work, size_t work_bytes,
                           hr_stream stream)
{
    return fermion_deriv(ctx, lat, m0, rep, gauge, X, L, coeff, force, 0, work, work_bytes, stream);
}

hr_status hr_fermion_link_grad(hr_ctx *ctx, hr_lattice lat, double m0, hr_rep rep, const void *gauge, const void *X,
                               const void *L, double coeff, double *grad, void *work, size_t work_bytes,
                               hr_stream stream)
{
    return fermion_deriv(ctx, lat, m0, rep, gauge, X, L, coeff, grad, 1, work, work_bytes, stream);
}

hr_status hr_force(hr_ctx *ctx, hr_lattice lat, const void *gauge, const void *a_full, const void *b_full,
                   double beta, double *force, hr_stream stream)
{
    return launch(ctx, lat, gauge, a_full, b_full, beta, force, 0, stream);
}

hr_status hr_link_grad(hr_ctx *ctx, hr_lattice lat, const void *a_full, const void *b_full, double beta,
                       double *grad, hr_stream stream)
{
    return launch(ctx, lat, nullptr, a_full, b_full, beta, grad, 1, stream);
}

} // extern "C"
