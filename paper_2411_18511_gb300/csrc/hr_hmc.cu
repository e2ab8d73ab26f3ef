// hr_hmc.cu -- hybrid Monte Carlo molecular dynamics for SU(2) with two
// flavours of even-odd preconditioned Wilson fermions in the fundamental
// representation (arXiv:2411.18511 Sec. 1 and Sec. 2.1 name the HMC as the
// consumer of the even-odd operator, its inverters and the fermion force).
//
// Conventions (the paper states none; the textbook scheme):
//   S_g = beta sum_{x, mu<nu} (1 - 1/2 Re tr P_mn(x))            (Wilson plaquette)
//   S_f = Re <eta, (Mhat^+ Mhat)^-1 eta>                          (pseudofermion, even sites)
//   momenta p_a(x, mu), a = 1..3; H = 1/2 sum p^2 + S_g + S_f
//   flow: U -> exp(i eps p.s/2) U,  p -> p - eps F,  F_a = dS/dw_a under U -> exp(i w.s/2) U
// The links are the caller's canonical quaternions (double[4][V][4],
// U = a0 + i a.s), updated in place; the momenta and forces are double[4][V][3].
//
// In quaternion form (a0 + i a.s)(b0 + i b.s) = (a0 b0 - a.b) + i(a0 b + b0 a - a x b).s,
// and a sum of SU(2) matrices keeps the form b0 + i b.s, so the staple sum V is
// a quaternion too.  The link U_mu(x) enters S_g as -beta/2 Re tr(U V) + const,
// and with W = U V = w0 + i w.s, Re tr((i s_a/2) W) = -w_a, so the gauge force
// is F_a = beta/2 w_a.  The fermion force is hr_force on the packed links
// (which carry the boundary conditions) with a = (Y, H_eo^+ Y), b = (X, H_oe X),
// X = (Mhat^+ Mhat)^-1 eta, Y = Mhat X, coefficient 2 / (4 (4 + m0)).
// Hasenbusch mass preconditioning splits S_f into Re<eta, (Mhat_H^+ Mhat_H)^-1 eta>
// (heavy mass m0_H) and Re<eta2, (Mhat^+ Mhat)^-1 eta2> with eta2 = Mhat_H^+ phi;
// the second term's force adds the variation of eta2: -2 c_H dRe<a', H b'>/dw,
// a' = (g5 X2, H_eo^+ g5 X2), b' = (g5 phi, H_oe g5 phi), c_H = 1/(4 (4 + m0_H)).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "hr_host.h"

using namespace hr;

namespace {

struct Qt {
    double w, x, y, z; // a0, a1, a2, a3
};
__device__ __forceinline__ Qt qmul(const Qt &a, const Qt &b)
{
    return {a.w * b.w - (a.x * b.x + a.y * b.y + a.z * b.z), a.w * b.x + b.w * a.x - (a.y * b.z - a.z * b.y),
            a.w * b.y + b.w * a.y - (a.z * b.x - a.x * b.z), a.w * b.z + b.w * a.z - (a.x * b.y - a.y * b.x)};
}
__device__ __forceinline__ Qt qconj(const Qt &a) { return {a.w, -a.x, -a.y, -a.z}; }
__device__ __forceinline__ Qt qadd(const Qt &a, const Qt &b) { return {a.w + b.w, a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ Qt qload(const double *q, long long V, int mu, long long x)
{
    const double *p = q + ((long long)mu * V + x) * 4;
    return {p[0], p[1], p[2], p[3]};
}

__device__ __forceinline__ void coords_of(const Geom &g, long long t, int (&x)[4])
{
    for (int k = 3; k >= 0; --k) {
        x[k] = (int)(t % g.d[k]);
        t /= g.d[k];
    }
}
__device__ __forceinline__ long long lex_at(const Geom &g, const int (&x)[4], int m1, int s1, int m2 = 0, int s2 = 0)
{
    int y[4] = {x[0], x[1], x[2], x[3]};
    y[m1] = (y[m1] + s1 + g.d[m1]) % g.d[m1];
    y[m2] = (y[m2] + s2 + g.d[m2]) % g.d[m2];
    return (((long long)y[0] * g.d[1] + y[1]) * g.d[2] + y[2]) * g.d[3] + y[3];
}

// block sum of v into partial[blockIdx.x] (blockDim.x = 256)
__device__ __forceinline__ void block_partial(double v, double *partial)
{
    __shared__ double sh[256];
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

constexpr int kRedBlocks = 1024; // grid of the reducing kernels (grid-stride loops)

// F[mu][x][a] += coeff * beta/2 * vec(U_mu(x) V_mu(x))_a, one thread per link
__global__ void k_gauge_force(Geom g, double beta, double coeff, const double *q, double *F)
{
    const long long V = 2LL * g.vh;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 4 * V) return;
    const int mu = (int)(t / V);
    const long long xl = t - (long long)mu * V;
    int x[4];
    coords_of(g, xl, x);
    Qt S = {0.0, 0.0, 0.0, 0.0};
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
        const long long xpm = lex_at(g, x, mu, 1), xpn = lex_at(g, x, nu, 1), xmn = lex_at(g, x, nu, -1);
        const long long xpm_mn = lex_at(g, x, mu, 1, nu, -1);
        // U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+  and  U_nu(x+mu-nu)^+ U_mu(x-nu)^+ U_nu(x-nu)
        S = qadd(S, qmul(qmul(qload(q, V, nu, xpm), qconj(qload(q, V, mu, xpn))), qconj(qload(q, V, nu, xl))));
        S = qadd(S, qmul(qmul(qconj(qload(q, V, nu, xpm_mn)), qconj(qload(q, V, mu, xmn))), qload(q, V, nu, xmn)));
    }
    const Qt W = qmul(qload(q, V, mu, xl), S);
    const double s = coeff * 0.5 * beta;
    double *f = F + t * 3;
    f[0] += s * W.x;
    f[1] += s * W.y;
    f[2] += s * W.z;
}

// partial sums of 1/2 tr P_mn(x) over mu < nu (the scalar part of the plaquette quaternion)
__global__ void __launch_bounds__(256) k_plaquette(Geom g, const double *q, double *partial)
{
    const long long V = 2LL * g.vh;
    double acc = 0.0;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < V; t += (long long)gridDim.x * blockDim.x) {
        int x[4];
        coords_of(g, t, x);
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = mu + 1; nu < 4; ++nu) {
                const Qt P = qmul(qmul(qload(q, V, mu, t), qload(q, V, nu, lex_at(g, x, mu, 1))),
                                  qconj(qmul(qload(q, V, nu, t), qload(q, V, mu, lex_at(g, x, nu, 1)))));
                acc += P.w;
            }
    }
    block_partial(acc, partial);
}

// U <- exp(i eps p.s/2) U = (cos th + i sin th n.s) U, th = eps |p| / 2, renormalised
__global__ void k_link_update(long long n_links, double eps, const double *p, double *q)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_links) return;
    const double *pp = p + t * 3;
    const double nrm = sqrt(pp[0] * pp[0] + pp[1] * pp[1] + pp[2] * pp[2]);
    const double th = 0.5 * eps * nrm;
    const double sn = nrm > 0.0 ? sin(th) / nrm : 0.0;
    const Qt E = {cos(th), sn * pp[0], sn * pp[1], sn * pp[2]};
    double *qq = q + t * 4;
    Qt U = qmul(E, {qq[0], qq[1], qq[2], qq[3]});
    const double inv = 1.0 / sqrt(U.w * U.w + U.x * U.x + U.y * U.y + U.z * U.z);
    qq[0] = U.w * inv;
    qq[1] = U.x * inv;
    qq[2] = U.y * inv;
    qq[3] = U.z * inv;
}

__global__ void k_axpy_d(long long n, double a, const double *x, double *y)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) y[t] += a * x[t];
}

__global__ void __launch_bounds__(256) k_sumsq(long long n, const double *x, double *partial)
{
    double acc = 0.0;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        acc += x[t] * x[t];
    block_partial(acc, partial);
}

// Re <a, b> of packed FP64 fundamental spinors of one parity
__global__ void __launch_bounds__(256) k_dot_re(Geom g, const void *a, const void *b, double *partial)
{
    double acc = 0.0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < g.vh; j += gridDim.x * blockDim.x) {
        cpx<dd> u[4][2], v[4][2];
        load_spinor<2, kF64>(a, g.nblk_s, j, u);
        load_spinor<2, kF64>(b, g.nblk_s, j, v);
        for (int s = 0; s < 4; ++s)
            for (int c = 0; c < 2; ++c)
                acc += dd_to_double(u[s][c].re) * dd_to_double(v[s][c].re) +
                       dd_to_double(u[s][c].im) * dd_to_double(v[s][c].im);
    }
    block_partial(acc, partial);
}

// sum the partials on the host, in block order (deterministic)
hr_status read_sum(hr_ctx *ctx, const double *partial, int n, double &out, cudaStream_t s)
{
    std::vector<double> h(n);
    cudaError_t e = cudaMemcpyAsync(h.data(), partial, sizeof(double) * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_error(ctx, HR_ERR_CUDA, "reduction readback: %s", cudaGetErrorString(e));
    double acc = 0.0;
    for (int k = 0; k < n; ++k) acc += h[k];
    out = acc;
    return HR_OK;
}

hr_status check_md(hr_ctx *ctx, hr_lattice lat)
{
    if (!ctx) return HR_ERR_INVALID_ARG;
    return validate_lattice(ctx, lat, 1);
}

hr_status gauge_force(hr_ctx *ctx, const Geom &g, double beta, const double *q, double coeff, double *F, cudaStream_t s)
{
    const long long n = 8LL * g.vh;
    k_gauge_force<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(g, beta, coeff, q, F);
    return check_launch(ctx, "gauge force");
}

// S_g and the average plaquette <1/2 tr P> over the 6 V plaquettes
hr_status gauge_action(hr_ctx *ctx, const Geom &g, double beta, const double *q, double &S, cudaStream_t s,
                       double *plaq = nullptr)
{
    k_plaquette<<<kRedBlocks, 256, 0, s>>>(g, q, ctx->d_partials);
    hr_status st = check_launch(ctx, "plaquette");
    double sum = 0.0;
    if (!st) st = read_sum(ctx, ctx->d_partials, kRedBlocks, sum, s);
    if (st) return st;
    const double n = 6.0 * 2.0 * g.vh;
    S = beta * (n - sum);
    if (plaq) *plaq = sum / n;
    return HR_OK;
}

hr_status kinetic(hr_ctx *ctx, const Geom &g, const double *p, double &K, cudaStream_t s)
{
    k_sumsq<<<kRedBlocks, 256, 0, s>>>(24LL * g.vh, p, ctx->d_partials);
    hr_status st = check_launch(ctx, "kinetic energy");
    double sum = 0.0;
    if (!st) st = read_sum(ctx, ctx->d_partials, kRedBlocks, sum, s);
    K = 0.5 * sum;
    return st;
}

hr_status link_update(hr_ctx *ctx, const Geom &g, double eps, const double *p, double *q, cudaStream_t s)
{
    const long long n = 8LL * g.vh;
    k_link_update<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(n, eps, p, q);
    return check_launch(ctx, "link update");
}

hr_status mom_update(hr_ctx *ctx, const Geom &g, double eps, const double *F, double *p, cudaStream_t s)
{
    const long long n = 24LL * g.vh;
    k_axpy_d<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, -eps, F, p);
    return check_launch(ctx, "momentum update");
}

// ---------------------------------------------------------------- trajectory

constexpr double kOmelyanLambda = 0.1931833275037836; // Omelyan's minimum-norm second-order scheme

struct HmcWork {
    void *gauge;      // packed FP64 fundamental links (with the boundary signs)
    double *F;        // force [4][V][3]
    double *Fg;       // gauge force of the inner level (two time scales)
    void *X;          // even half: (Mhat^+ Mhat)^-1 eta (Hasenbusch: at the heavy mass)
    void *X2, *eta2;  // Hasenbusch ratio term: eta2 = Mhat_H^+ phi, X2 = (Mhat^+ Mhat)^-1 eta2
    void *e1, *e2;    // even temporaries (g5 copies)
    void *a, *b;      // full fields of the fermion force
    void *t_odd;      // odd temporary of Mhat
    void *cg;         // CG workspace
    size_t cg_bytes;
    void *clover;     // clover fermions: the packed FP64 clover field of the current links
    void *clover_h;   // with Hasenbusch: the clover field at the heavy mass
    void *cf;         // clover force workspace
    size_t cf_bytes;
};

// two time scales: the fermion integrator's link updates run inner gauge steps
bool nested(const hr_hmc_params &prm) { return prm.fermions && prm.n_steps_gauge > 1; }

size_t layout_hmc(hr_lattice lat, const hr_hmc_params &prm, char *w, HmcWork *hw)
{
    const size_t half = hr_spinor_packed_bytes(lat, HR_FUND, HR_F64, HR_EVEN, 1);
    const size_t gb = hr_gauge_packed_bytes(lat, HR_FUND, HR_F64);
    hr_solver_opts o = prm.solver;
    o.n_rhs = 1;
    o.x0_is_guess = 0;
    size_t cgb = hr_cg_workspace_bytes(lat, HR_FUND, &o);
    if (prm.clover) cgb = std::max(cgb, hr_cg_clover_workspace_bytes(lat, HR_FUND, &o));
    const long long V = (long long)lat.dims[0] * lat.dims[1] * lat.dims[2] * lat.dims[3];
    size_t off = 0;
    auto take = [&](size_t n) -> void * {
        void *p = w ? (void *)(w + off) : nullptr;
        off += (n + 255) & ~(size_t)255;
        return p;
    };
    void *gauge = take(gb);
    void *F = take(sizeof(double) * 12 * V);
    void *Fg = nested(prm) ? take(sizeof(double) * 12 * V) : nullptr;
    void *X = take(half), *a = take(2 * half), *b = take(2 * half), *t = take(half);
    void *X2 = nullptr, *eta2 = nullptr, *e1 = nullptr, *e2 = nullptr;
    if (prm.hasenbusch) {
        X2 = take(half);
        eta2 = take(half);
        e1 = take(half);
        e2 = take(half);
    }
    void *cg = take(cgb);
    void *clover = nullptr, *clover_h = nullptr, *cf = nullptr;
    size_t cfb = 0;
    if (prm.clover) {
        clover = take(hr_clover_packed_bytes(lat, HR_FUND, HR_F64));
        if (prm.hasenbusch) clover_h = take(hr_clover_packed_bytes(lat, HR_FUND, HR_F64));
        cfb = hr_clover_force_workspace_bytes(lat);
        cf = take(cfb);
    }
    if (hw)
        *hw = HmcWork{gauge, (double *)F, (double *)Fg, X, X2, eta2, e1, e2, a, b, t, cg, cgb, clover, clover_h, cf,
                      cfb};
    return off;
}

struct Trajectory {
    hr_ctx *ctx;
    hr_lattice lat;
    Geom g;
    hr_hmc_params prm;
    double *q;
    double *p;
    const void *eta;
    const void *phi;  // Hasenbusch ratio pseudofermion (nullptr without)
    HmcWork w;
    cudaStream_t s;
    size_t half;
    bool force_valid = false; // F holds the force of the current links
    bool x_valid = false;     // X holds the solve of the current links
    int cg_iters = 0, solves = 0;

    hr_status pack() { return hr_gauge_pack(ctx, lat, HR_FUND, HR_F64, q, w.gauge, (hr_stream)s); }

    // the mass of the solve with eta: the heavy one under Hasenbusch preconditioning
    double eta_mass() const { return prm.hasenbusch ? prm.m0_hasenbusch : prm.m0; }

    // the clover field of a solve at mass m0 (the heavy one under Hasenbusch)
    void *clover_of(double m0) const
    {
        return (prm.hasenbusch && m0 == prm.m0_hasenbusch && m0 != prm.m0) ? w.clover_h : w.clover;
    }

    hr_status cg(double m0, const void *src, void *x)
    {
        hr_solver_opts o = prm.solver;
        o.n_rhs = 1;
        o.x0_is_guess = 0;
        hr_solve_info info{};
        hr_status st = prm.clover ? hr_cg_solve_clover(ctx, lat, HR_FUND, &o, w.gauge, clover_of(m0), src, x, &info,
                                                       w.cg, w.cg_bytes, (hr_stream)s)
                                  : hr_cg_solve(ctx, lat, m0, HR_FUND, &o, w.gauge, src, x, &info, w.cg, w.cg_bytes,
                                                (hr_stream)s);
        cg_iters += info.iters;
        ++solves;
        return st;
    }

    hr_status solve()
    {
        if (x_valid) return HR_OK;
        hr_status st = pack();
        if (!st && prm.clover)
            st = hr_clover_build(ctx, lat, HR_FUND, HR_F64, prm.clover_kind, prm.m0, prm.c_sw, q, w.clover,
                                 (hr_stream)s);
        if (!st && prm.clover && prm.hasenbusch)
            st = hr_clover_build(ctx, lat, HR_FUND, HR_F64, prm.clover_kind, prm.m0_hasenbusch, prm.c_sw, q,
                                 w.clover_h, (hr_stream)s);
        if (!st) st = cg(eta_mass(), eta, w.X);
        if (!st && prm.hasenbusch) {
            // eta2 = Mhat_H^+ phi at the current links, then the ratio term's solve
            st = apply_eo_op(ctx, g, prm.m0_hasenbusch, HR_FUND, kF64, HR_OP_SCHUR_DAG, w.gauge, phi, w.eta2,
                             w.t_odd, nullptr, kFinNone, nullptr, nullptr, s, nullptr,
                             prm.clover ? w.clover_h : nullptr);
            if (!st) st = cg(prm.m0, w.eta2, w.X2);
        }
        if (st) return st;
        x_valid = true;
        return HR_OK;
    }

    hr_status dot(const void *a, const void *b, double &out)
    {
        k_dot_re<<<kRedBlocks, 256, 0, s>>>(g, a, b, ctx->d_partials);
        hr_status st = check_launch(ctx, "pseudofermion action");
        if (!st) st = read_sum(ctx, ctx->d_partials, kRedBlocks, out, s);
        return st;
    }

    hr_status fermion_action(double &S)
    {
        hr_status st = solve();
        if (!st) st = dot(eta, w.X, S);
        if (!st && prm.clover) {
            // S_det = -2 sum_{odd} log det A
            double ld = 0.0;
            st = hr_clover_logdet(ctx, lat, HR_FUND, w.clover, HR_ODD, &ld, (hr_stream)s);
            S += -2.0 * ld;
        }
        if (!st && prm.hasenbusch) {
            double S2 = 0.0;
            st = dot(w.eta2, w.X2, S2);
            S += S2;
        }
        return st;
    }

    hr_status copy(void *dst, const void *src)
    {
        cudaError_t e = cudaMemcpyAsync(dst, src, half, cudaMemcpyDeviceToDevice, s);
        return e == cudaSuccess ? HR_OK : set_error(ctx, HR_ERR_CUDA, "copy: %s", cudaGetErrorString(e));
    }

    // dst_odd = [g5] H_oe [g5] src_even (g5 on the input and / or the output)
    hr_status hop_oe(const void *src, void *dst, int g5_in, int g5_out)
    {
        HopLaunch L{};
        L.p = 1;
        L.gauge = w.gauge;
        L.in = src;
        L.out = dst;
        L.beta = 1.0;
        L.g5_in = g5_in;
        L.g5_out = g5_out;
        return launch_hop(ctx, g, HR_FUND, kF64, L, s);
    }

    // F += coeff dRe<a, H b>/dw with a = (u, H_eo^+ u), b = (v, H_oe v), H_eo^+ = g5 H_oe g5
    hr_status pair_force(const void *u, const void *v, double coeff)
    {
        char *a = (char *)w.a, *b = (char *)w.b;
        hr_status st = copy(a, u);
        if (!st) st = hop_oe(u, a + half, 1, 1);
        if (!st) st = copy(b, v);
        if (!st) st = hop_oe(v, b + half, 0, 0);
        if (!st) st = hr_force(ctx, lat, w.gauge, a, b, coeff, w.F, (hr_stream)s);
        return st;
    }

    // the force of Re<src, (Mhat^+ Mhat)^-1 src> at mass m0 with X its solution:
    // 2c dRe<a, H b>/dw, a = (Mhat X, H_eo^+ Mhat X), b = (X, H_oe X), c = 1/(4 (4+m0))
    hr_status solve_force(double m0, const void *X)
    {
        hr_status st = apply_eo_op(ctx, g, m0, HR_FUND, kF64, HR_OP_SCHUR, w.gauge, X, w.a, w.t_odd, nullptr,
                                   kFinNone, nullptr, nullptr, s);
        if (st) return st;
        char *a = (char *)w.a, *b = (char *)w.b; // Mhat X is a's even half already
        st = hop_oe(a, a + half, 1, 1);
        if (!st) st = copy(b, X);
        if (!st) st = hop_oe(X, b + half, 0, 0);
        if (!st) st = hr_force(ctx, lat, w.gauge, a, b, 2.0 / (4.0 * (4.0 + m0)), w.F, (hr_stream)s);
        return st;
    }

    hr_status zero(double *F)
    {
        cudaError_t e = cudaMemsetAsync(F, 0, sizeof(double) * 24 * g.vh, s);
        return e == cudaSuccess ? HR_OK : set_error(ctx, HR_ERR_CUDA, "force reset: %s", cudaGetErrorString(e));
    }

    // F = the gauge force plus the pseudofermion force of the current links
    hr_status force()
    {
        if (force_valid) return HR_OK;
        hr_status st = zero(w.F);
        if (!st) st = gauge_force(ctx, g, prm.beta, q, 1.0, w.F, s);
        if (!st) st = fermion_terms();
        if (!st) force_valid = true;
        return st;
    }

    // F += the pseudofermion force of the current links
    hr_status fermion_terms()
    {
        hr_status st = HR_OK;
        if (prm.fermions && prm.clover) {
            auto cforce = [&](double m0, const void *clov, const void *X, const void *Y, int det, double coeff) {
                return hr_clover_fermion_force(ctx, lat, prm.clover_kind, m0, prm.c_sw, q, w.gauge, clov, X, Y, det,
                                               coeff, w.F, w.cf, w.cf_bytes, (hr_stream)s);
            };
            st = solve();
            if (!prm.hasenbusch) {
                if (!st) st = cforce(prm.m0, w.clover, w.X, nullptr, 1, 1.0);
            } else {
                // heavy term; ratio term's solve (and the light det A_oo); the variation of
                // eta2 = Mhat_H^+ phi: 2 Re<phi, dMhat_H X2>, minus the force of -2 Re<Y, dMhat_H X>
                if (!st) st = cforce(prm.m0_hasenbusch, w.clover_h, w.X, nullptr, 0, 1.0);
                if (!st) st = cforce(prm.m0, w.clover, w.X2, nullptr, 1, 1.0);
                if (!st) st = cforce(prm.m0_hasenbusch, w.clover_h, w.X2, phi, 0, -1.0);
            }
        } else if (prm.fermions) {
            st = solve();
            if (!st) st = solve_force(eta_mass(), w.X);
            if (!st && prm.hasenbusch) {
                // the ratio term: its solve's force, and the variation of eta2 = Mhat_H^+ phi,
                // -2 c_H dRe<a', H b'>/dw with a' = (g5 X2, H_eo^+ g5 X2), b' = (g5 phi, H_oe g5 phi)
                st = solve_force(prm.m0, w.X2);
                if (!st) st = copy(w.e1, w.X2);
                if (!st) st = blas_gamma5(ctx, g, HR_FUND, w.e1, s);
                if (!st) st = copy(w.e2, phi);
                if (!st) st = blas_gamma5(ctx, g, HR_FUND, w.e2, s);
                if (!st) st = pair_force(w.e1, w.e2, -2.0 / (4.0 * (4.0 + prm.m0_hasenbusch)));
            }
        }
        return st;
    }

    hr_status kick(double eps)
    {
        hr_status st = force();
        if (!st) st = mom_update(ctx, g, eps, w.F, p, s);
        return st;
    }

    hr_status drift(double eps)
    {
        force_valid = ferm_valid = gauge_valid = false;
        x_valid = false;
        return link_update(ctx, g, eps, p, q, s);
    }

    // ---- two time scales (n_steps_gauge > 1): F holds the pseudofermion
    // force alone, Fg the gauge force, each reused until the links move
    bool ferm_valid = false, gauge_valid = false;

    hr_status kick_fermion(double eps)
    {
        hr_status st = HR_OK;
        if (!ferm_valid) {
            st = zero(w.F);
            if (!st) st = fermion_terms();
            if (!st) ferm_valid = true;
        }
        if (!st) st = mom_update(ctx, g, eps, w.F, p, s);
        return st;
    }

    hr_status kick_gauge(double eps)
    {
        hr_status st = HR_OK;
        if (!gauge_valid) {
            st = zero(w.Fg);
            if (!st) st = gauge_force(ctx, g, prm.beta, q, 1.0, w.Fg, s);
            if (!st) gauge_valid = true;
        }
        if (!st) st = mom_update(ctx, g, eps, w.Fg, p, s);
        return st;
    }

    // one step of length eps of the integrator with the given kick and drift
    template <class Kick, class Drift> hr_status step(double eps, Kick kick_fn, Drift drift_fn)
    {
        hr_status st;
        if (prm.integrator == HR_INTEGRATOR_LEAPFROG) {
            st = kick_fn(0.5 * eps);
            if (!st) st = drift_fn(eps);
            if (!st) st = kick_fn(0.5 * eps);
        } else {
            const double lam = kOmelyanLambda;
            st = kick_fn(lam * eps);
            if (!st) st = drift_fn(0.5 * eps);
            if (!st) st = kick_fn((1.0 - 2.0 * lam) * eps);
            if (!st) st = drift_fn(0.5 * eps);
            if (!st) st = kick_fn(lam * eps);
        }
        return st;
    }

    // the outer level's link update of length t: n_steps_gauge gauge steps
    hr_status inner(double t)
    {
        const int m = prm.n_steps_gauge;
        hr_status st = HR_OK;
        for (int j = 0; j < m && !st; ++j)
            st = step(t / m, [&](double e) { return kick_gauge(e); }, [&](double e) { return drift(e); });
        return st;
    }

    double plaq = 0.0;

    hr_status hamiltonian(double &K, double &Sg, double &Sf)
    {
        hr_status st = kinetic(ctx, g, p, K, s);
        if (!st) st = gauge_action(ctx, g, prm.beta, q, Sg, s, &plaq);
        Sf = 0.0;
        if (!st && prm.fermions) st = fermion_action(Sf);
        return st;
    }
};

} // namespace

extern "C" {

hr_status hr_gauge_force(hr_ctx *ctx, hr_lattice lat, double beta, const double *gauge, double coeff, double *force,
                         hr_stream stream)
{
    hr_status st = check_md(ctx, lat);
    if (st) return st;
    st = check_buffers(ctx, {}, {gauge, force});
    if (st) return st;
    return gauge_force(ctx, make_geom(lat, 1), beta, gauge, coeff, force, (cudaStream_t)stream);
}

hr_status hr_gauge_action(hr_ctx *ctx, hr_lattice lat, double beta, const double *gauge, double *action,
                          hr_stream stream)
{
    hr_status st = check_md(ctx, lat);
    if (st) return st;
    if (!action) return set_error(ctx, HR_ERR_INVALID_ARG, "null result pointer");
    st = check_buffers(ctx, {}, {gauge});
    if (st) return st;
    return gauge_action(ctx, make_geom(lat, 1), beta, gauge, *action, (cudaStream_t)stream);
}

hr_status hr_link_update(hr_ctx *ctx, hr_lattice lat, double eps, const double *mom, double *gauge, hr_stream stream)
{
    hr_status st = check_md(ctx, lat);
    if (st) return st;
    st = check_buffers(ctx, {}, {mom, gauge});
    if (st) return st;
    return link_update(ctx, make_geom(lat, 1), eps, mom, gauge, (cudaStream_t)stream);
}

hr_status hr_mom_update(hr_ctx *ctx, hr_lattice lat, double eps, const double *force, double *mom, hr_stream stream)
{
    hr_status st = check_md(ctx, lat);
    if (st) return st;
    st = check_buffers(ctx, {}, {force, mom});
    if (st) return st;
    return mom_update(ctx, make_geom(lat, 1), eps, force, mom, (cudaStream_t)stream);
}

hr_status hr_kinetic_energy(hr_ctx *ctx, hr_lattice lat, const double *mom, double *energy, hr_stream stream)
{
    hr_status st = check_md(ctx, lat);
    if (st) return st;
    if (!energy) return set_error(ctx, HR_ERR_INVALID_ARG, "null result pointer");
    st = check_buffers(ctx, {}, {mom});
    if (st) return st;
    return kinetic(ctx, make_geom(lat, 1), mom, *energy, (cudaStream_t)stream);
}

size_t hr_hmc_workspace_bytes(hr_lattice lat, const hr_hmc_params *prm)
{
    if (!prm || hr_gauge_packed_bytes(lat, HR_FUND, HR_F64) == 0) return 0;
    hr_solver_opts o = prm->solver;
    o.n_rhs = 1;
    if (hr_cg_workspace_bytes(lat, HR_FUND, &o) == 0) return 0;
    return layout_hmc(lat, *prm, nullptr, nullptr);
}

hr_status hr_hmc_trajectory(hr_ctx *ctx, hr_lattice lat, const hr_hmc_params *prm, double *gauge, double *mom,
                            const void *eta, const void *phi, hr_hmc_info *info, void *work, size_t work_bytes,
                            hr_stream stream)
{
    if (!ctx) return HR_ERR_INVALID_ARG;
    if (info) std::memset(info, 0, sizeof *info);
    if (!prm) return set_error(ctx, HR_ERR_INVALID_ARG, "null parameters");
    hr_status st = validate_lattice(ctx, lat, 1);
    if (st) return st;
    if (prm->n_steps < 1 || !(prm->tau > 0.0) || !std::isfinite(prm->beta) || !std::isfinite(prm->tau))
        return set_error(ctx, HR_ERR_INVALID_ARG, "n_steps >= 1, tau > 0 and a finite beta are needed");
    if (prm->integrator != HR_INTEGRATOR_LEAPFROG && prm->integrator != HR_INTEGRATOR_OMELYAN)
        return set_error(ctx, HR_ERR_INVALID_ARG, "bad integrator");
    if (prm->fermions && !(4.0 + prm->m0 != 0.0)) return set_error(ctx, HR_ERR_INVALID_ARG, "4 + m0 must be nonzero");
    if (prm->fermions && prm->hasenbusch && !(4.0 + prm->m0_hasenbusch != 0.0))
        return set_error(ctx, HR_ERR_INVALID_ARG, "4 + m0_hasenbusch must be nonzero");
    if (prm->hasenbusch && !prm->fermions) return set_error(ctx, HR_ERR_INVALID_ARG, "Hasenbusch needs fermions");
    if (prm->clover && (!prm->fermions || !std::isfinite(prm->c_sw) ||
                        (prm->clover_kind != HR_CLOVER_SW && prm->clover_kind != HR_CLOVER_EXP)))
        return set_error(ctx, HR_ERR_INVALID_ARG, "clover fermions: fermions on, a kind, a finite c_sw");
    if (prm->clover && prm->hasenbusch && prm->m0_hasenbusch == prm->m0)
        return set_error(ctx, HR_ERR_INVALID_ARG, "Hasenbusch needs a heavy mass other than m0");
    if (prm->n_steps_gauge < 0 || prm->n_steps_gauge > 1000)
        return set_error(ctx, HR_ERR_INVALID_ARG, "n_steps_gauge must lie in [0, 1000]");
    if (prm->fermions && prm->hasenbusch) st = check_buffers(ctx, {eta, phi}, {gauge, mom}, {work});
    else if (prm->fermions) st = check_buffers(ctx, {eta}, {gauge, mom}, {work});
    else st = check_buffers(ctx, {}, {gauge, mom}, {work});
    if (st) return st;
    const size_t need = hr_hmc_workspace_bytes(lat, prm);
    if (need == 0) return set_error(ctx, HR_ERR_INVALID_ARG, "bad solver options");
    if (!work || work_bytes < need)
        return set_error(ctx, HR_ERR_WORKSPACE, "workspace of %zu bytes needed, %zu given", need, work_bytes);

    const auto t0 = std::chrono::steady_clock::now();
    Trajectory T;
    T.ctx = ctx;
    T.lat = lat;
    T.g = make_geom(lat, 1);
    T.prm = *prm;
    T.q = gauge;
    T.p = mom;
    T.eta = eta;
    T.phi = prm->hasenbusch ? phi : nullptr;
    T.s = (cudaStream_t)stream;
    T.half = hr_spinor_packed_bytes(lat, HR_FUND, HR_F64, HR_EVEN, 1);
    layout_hmc(lat, *prm, (char *)work, &T.w);

    double K0, Sg0, Sf0, K1, Sg1, Sf1;
    st = T.hamiltonian(K0, Sg0, Sf0);
    const double eps = prm->tau / prm->n_steps;
    const bool two_scales = nested(*prm);
    for (int k = 0; k < prm->n_steps && !st; ++k) {
        if (two_scales)
            st = T.step(eps, [&](double e) { return T.kick_fermion(e); }, [&](double e) { return T.inner(e); });
        else
            st = T.step(eps, [&](double e) { return T.kick(e); }, [&](double e) { return T.drift(e); });
    }
    if (!st) st = T.hamiltonian(K1, Sg1, Sf1);
    if (st) return st;
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (info) {
        info->dH = (K1 + Sg1 + Sf1) - (K0 + Sg0 + Sf0);
        info->kinetic_start = K0;
        info->kinetic_end = K1;
        info->gauge_action_start = Sg0;
        info->gauge_action_end = Sg1;
        info->fermion_action_start = Sf0;
        info->fermion_action_end = Sf1;
        info->plaquette = T.plaq;
        info->cg_iters = T.cg_iters;
        info->solves = T.solves;
        info->seconds = secs;
    }
    if (!std::isfinite(K1 + Sg1 + Sf1)) return set_error(ctx, HR_ERR_NUMERIC, "NaN or Inf in the Hamiltonian");
    return HR_OK;
}

} // extern "C"
