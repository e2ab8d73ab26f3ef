// hr_cg.cu -- conjugate-gradient solvers on the even-odd normal operator
// A = Mhat^+ Mhat (even sites), the "inverters" of arXiv:2411.18511 Sec. 1
// applied to the even-odd preconditioned operator of Sec. 2.1.
//
// * FP64 CG (Hestenes-Stiefel).  One iteration is four hop launches (the
//   second one reduces |Mhat p|^2 = <p, A p> and sets alpha on the device),
//   one fused x/r update with the |r|^2 reduction (sets beta and the per-RHS
//   convergence flags on the device) and one p update.  No host round trip per
//   iteration: a chunk of iterations is captured once into a CUDA graph and
//   replayed; the host reads the device flags once per chunk.
// * Mixed precision with reliable updates (Clark et al., Comput. Phys. Commun.
//   181 (2010) 1517): the recurrence runs on FP32 or FP16 copies of the gauge
//   field and of p, r, q with FP32 arithmetic and an FP32 solution increment.
//   When |r| drops below delta * max|r| since the last update (or below the
//   target), a device-gated block adds the increment into the FP64 solution,
//   recomputes r = b - A x in FP64 and restarts the low-precision residual from
//   it, keeping the search direction.  Convergence is only declared on an FP64
//   residual.
// * n_rhs independent right-hand sides run as one "virtual site" field: every
//   link load serves all of them, and alpha, beta and convergence are per RHS.
#include <cmath>
#include <cstring>
#include <vector>

#include "hr_host.h"

using namespace hr;

namespace {

struct Graph {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t e = nullptr;
    ~Graph()
    {
        if (e) cudaGraphExecDestroy(e);
        if (g) cudaGraphDestroy(g);
    }
};

hr_status cuda_err(hr_ctx *ctx, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return HR_OK;
    cudaGetLastError();
    return set_error(ctx, HR_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

hr_status init_scalars(hr_ctx *ctx, int nrhs, double tol, double delta, cudaStream_t s)
{
    std::vector<double> h(kScalDoubles, 0.0);
    for (int r = 0; r < nrhs; ++r) h[S_ACTIVE * kMaxRhsSlots + r] = 1.0;
    h[S_DELTA2 * kMaxRhsSlots + 0] = delta * delta;
    h[S_DELTA2 * kMaxRhsSlots + 1] = tol * tol;
    std::memcpy(ctx->h_scal, h.data(), sizeof(double) * kScalDoubles);
    cudaError_t e = cudaMemcpyAsync(ctx->d_scal, ctx->h_scal, sizeof(double) * kScalDoubles, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return cuda_err(ctx, e, "scalar init");
}

// copy `n` slots of kMaxRhsSlots doubles starting at slot `first` to ctx->h_scal
hr_status read_scalars(hr_ctx *ctx, int first, int n, cudaStream_t s)
{
    cudaError_t e = cudaMemcpyAsync(ctx->h_scal, ctx->d_scal + first * kMaxRhsSlots,
                                    sizeof(double) * kMaxRhsSlots * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return cuda_err(ctx, e, "scalar readback");
}

inline const double *flag_ptr(hr_ctx *ctx, int f) { return ctx->d_scal + S_FLAGS * kMaxRhsSlots + f; }

struct Solver {
    hr_ctx *ctx;
    Geom g;
    double m0;
    int rep;
    hr_solver_opts o;
    const void *gauge;
    const void *b;
    void *x;
    cudaStream_t s;
    // FP64 buffers
    void *r64, *p64, *q64, *u64, *t64;
    // low precision buffers
    void *gauge_lo, *r_lo, *p_lo, *q_lo, *u_lo, *t_lo, *x_lo;
    size_t h64, hlo, h32, glo;

    bool mixed() const { return o.inner_prec != HR_F64; }

    static size_t layout(const Geom &g, int rep, const hr_solver_opts &o, Solver *sv, void *work)
    {
        size_t h64 = spinor_half_bytes(g, rep, kF64);
        char *w = (char *)work;
        size_t off = 0;
        auto take = [&](size_t n) -> void * {
            void *p = w ? (void *)(w + off) : nullptr;
            off += (n + 255) & ~(size_t)255;
            return p;
        };
        if (o.inner_prec == HR_F64) {
            void *r = take(h64), *p = take(h64), *q = take(h64), *u = take(h64), *t = take(h64);
            if (sv) {
                sv->r64 = r; sv->p64 = p; sv->q64 = q; sv->u64 = u; sv->t64 = t;
                sv->h64 = h64;
            }
        } else {
            size_t hlo = spinor_half_bytes(g, rep, o.inner_prec);
            size_t h32 = spinor_half_bytes(g, rep, kF32);
            size_t glo = gauge_bytes(g, rep, o.inner_prec);
            // the gauge is shared by all RHS: size it with one RHS
            void *r = take(h64), *q = take(h64), *u = take(h64), *t = take(h64);
            void *gl = take(glo), *rl = take(hlo), *pl = take(hlo), *ql = take(hlo), *ul = take(hlo), *tl = take(hlo);
            void *xl = take(h32);
            if (sv) {
                sv->r64 = r; sv->q64 = q; sv->u64 = u; sv->t64 = t; sv->p64 = nullptr;
                sv->gauge_lo = gl; sv->r_lo = rl; sv->p_lo = pl; sv->q_lo = ql; sv->u_lo = ul; sv->t_lo = tl;
                sv->x_lo = xl;
                sv->h64 = h64; sv->hlo = hlo; sv->h32 = h32; sv->glo = glo;
            }
        }
        return off;
    }

    // ax = A v in FP64 (gated launches skip unless *gate != 0)
    hr_status apply64(const void *v, void *ax, int fin, const double *gate, const double *done)
    {
        return apply_eo_op(ctx, g, m0, rep, kF64, HR_OP_NORMAL, gauge, v, ax, t64, u64, fin, gate, done, s);
    }

    hr_status iteration()
    {
        hr_status st;
        const double *done = flag_ptr(ctx, F_DONE);
        if (!mixed()) {
            st = apply64(p64, q64, kFinAlpha, nullptr, done);
            if (!st) st = blas_xr(ctx, g, rep, kF64, kF64, kF64, kF64, x, p64, r64, q64, s);
            if (!st) st = blas_p(ctx, g, rep, kF64, kF64, p64, r64, s);
            return st;
        }
        const int P = o.inner_prec;
        Geom g1 = g; // the low-precision gauge is indexed like any gauge
        st = apply_eo_op(ctx, g1, m0, rep, P, HR_OP_NORMAL, gauge_lo, p_lo, q_lo, t_lo, u_lo, kFinAlpha, nullptr,
                         done, s);
        if (!st) st = blas_xr(ctx, g, rep, kF32, P, P, P, x_lo, p_lo, r_lo, q_lo, s);
        // reliable update, gated on the device
        const double *gate = flag_ptr(ctx, F_GATE);
        if (!st) st = blas_accum(ctx, g, rep, kF32, x, x_lo, gate, s);
        if (!st) st = apply64(x, q64, kFinNone, gate, nullptr);
        if (!st) st = blas_residual(ctx, g, rep, b, q64, r64, kFinResidual, gate, P, r_lo, s);
        if (!st) st = blas_p(ctx, g, rep, P, P, p_lo, r_lo, s);
        return st;
    }

    // r = b - A x (FP64), |r|^2 -> fin; for mixed also r_lo
    hr_status true_residual(int fin)
    {
        hr_status st = apply64(x, q64, kFinNone, nullptr, nullptr);
        if (st) return st;
        return blas_residual(ctx, g, rep, b, q64, r64, fin, nullptr, mixed() ? o.inner_prec : kF64,
                             mixed() ? r_lo : nullptr, s);
    }

    hr_status start()
    {
        hr_status st = init_scalars(ctx, g.nrhs, o.tol, o.reliable_delta, s);
        if (st) return st;
        if (mixed()) {
            st = gauge_convert(ctx, make_geom_gauge(), rep, o.inner_prec, gauge, gauge_lo, s);
            if (st) return st;
        }
        st = blas_norm2(ctx, g, rep, kF64, b, kFinBB, s);
        if (st) return st;
        if (o.x0_is_guess) {
            st = true_residual(kFinInit);
        } else {
            st = blas_zero(ctx, g, rep, kF64, x, s);
            if (!st) st = blas_copy(ctx, g, rep, kF64, b, r64, s);
            if (!st) st = blas_norm2(ctx, g, rep, kF64, r64, kFinInit, s);
            if (!st && mixed()) st = blas_convert(ctx, g, rep, kF64, o.inner_prec, r64, r_lo, nullptr, s);
        }
        if (st) return st;
        return restart_direction();
    }

    hr_status restart_direction()
    {
        if (!mixed()) return blas_copy(ctx, g, rep, kF64, r64, p64, s);
        hr_status st = blas_zero(ctx, g, rep, kF32, x_lo, s);
        if (!st) st = blas_copy(ctx, g, rep, o.inner_prec, r_lo, p_lo, s);
        return st;
    }

    Geom make_geom_gauge() const { return g; }
};

} // namespace

extern "C" {

hr_solver_opts hr_solver_default_opts(void)
{
    hr_solver_opts o;
    o.tol = 1e-10;
    o.maxiter = 20000;
    o.inner_prec = HR_F64;
    o.reliable_delta = 0.1;
    o.n_rhs = 1;
    o.x0_is_guess = 0;
    o.check_every = 0;
    return o;
}

size_t hr_cg_workspace_bytes(hr_lattice lat, hr_rep rep, const hr_solver_opts *opts)
{
    if (!opts || !valid_rep(rep) || !valid_prec(opts->inner_prec) || opts->n_rhs < 1 || opts->n_rhs > kMaxRhs)
        return 0;
    if (hr_spinor_packed_bytes(lat, rep, HR_F64, HR_EVEN, opts->n_rhs) == 0) return 0;
    return Solver::layout(make_geom(lat, opts->n_rhs), rep, *opts, nullptr, nullptr);
}

hr_status hr_cg_solve(hr_ctx *ctx, hr_lattice lat, double m0, hr_rep rep, const hr_solver_opts *opts,
                      const void *gauge, const void *b, void *x, hr_solve_info *info, void *work, size_t work_bytes,
                      hr_stream stream)
{
    if (!ctx) return HR_ERR_INVALID_ARG;
    if (info) std::memset(info, 0, sizeof *info);
    if (!opts) return set_error(ctx, HR_ERR_INVALID_ARG, "null options");
    if (!valid_rep(rep)) return set_error(ctx, HR_ERR_INVALID_ARG, "bad rep");
    if (!valid_prec(opts->inner_prec)) return set_error(ctx, HR_ERR_INVALID_ARG, "bad inner precision");
    if (!(opts->tol > 0.0) || opts->maxiter < 1) return set_error(ctx, HR_ERR_INVALID_ARG, "tol must be > 0 and maxiter >= 1");
    if (opts->inner_prec != HR_F64 && !(opts->reliable_delta > 0.0 && opts->reliable_delta < 1.0))
        return set_error(ctx, HR_ERR_INVALID_ARG, "reliable_delta must lie in (0, 1)");
    hr_status st = validate_lattice(ctx, lat, opts->n_rhs);
    if (st) return st;
    if (!gauge || !b || !x) return set_error(ctx, HR_ERR_INVALID_ARG, "null field pointer");
    if (b == x) return set_error(ctx, HR_ERR_INVALID_ARG, "b and x must not alias");
    if (!(4.0 + m0 != 0.0)) return set_error(ctx, HR_ERR_INVALID_ARG, "4 + m0 must be nonzero");
    size_t need = hr_cg_workspace_bytes(lat, rep, opts);
    if (!work || work_bytes < need)
        return set_error(ctx, HR_ERR_WORKSPACE, "workspace of %zu bytes needed, %zu given", need, work_bytes);

    Solver sv{};
    sv.ctx = ctx;
    sv.g = make_geom(lat, opts->n_rhs);
    sv.m0 = m0;
    sv.rep = rep;
    sv.o = *opts;
    sv.gauge = gauge;
    sv.b = b;
    sv.x = x;
    sv.s = (cudaStream_t)stream;
    Solver::layout(sv.g, rep, *opts, &sv, work);
    cudaStream_t s = sv.s;

    cudaError_t e = cudaEventRecord(ctx->ev0, s);
    if (e != cudaSuccess) return cuda_err(ctx, e, "event record");
    st = sv.start();
    if (st) return st;

    // capture `chunk` iterations once, replay the graph
    int chunk = opts->check_every > 0 ? opts->check_every : 16;
    if (chunk > opts->maxiter) chunk = opts->maxiter;
    // The graph bakes in every launch parameter: buffers, lattice, m0, the hop
    // shapes in use.  Solves that repeat them (a benchmark, an MD trajectory
    // with persistent buffers) reuse the instantiated graph from the context.
    char keybuf[512];
    {
        HopChoice c64 = hop_choice(ctx, sv.g, rep, kF64), clo = hop_choice(ctx, sv.g, rep, opts->inner_prec);
        unsigned long long m0bits;
        std::memcpy(&m0bits, &m0, sizeof m0bits);
        snprintf(keybuf, sizeof keybuf, "cg:%d:%d:%d:%d:%d:%d:%d:%llx:%d:%d:%p:%p:%p:%p:%d.%d:%d.%d:%zu", lat.dims[0],
                 lat.dims[1], lat.dims[2], lat.dims[3], sv.g.nrhs, rep, opts->inner_prec, m0bits, chunk,
                 (int)sizeof(void *), gauge, b, x, work, c64.variant, c64.block, clo.variant, clo.block, work_bytes);
    }
    cudaGraphExec_t exec = nullptr;
    auto cached = ctx->graphs.find(keybuf);
    if (cached != ctx->graphs.end()) {
        exec = cached->second.second;
    } else {
        Graph G;
        cudaStream_t cs;
        e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_err(ctx, e, "capture stream");
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            cudaStreamDestroy(cs);
            return cuda_err(ctx, e, "begin capture");
        }
        sv.s = cs;
        for (int k = 0; k < chunk && !st; ++k) st = sv.iteration();
        sv.s = s;
        cudaError_t e2 = cudaStreamEndCapture(cs, &G.g);
        cudaStreamDestroy(cs);
        if (st) return st;
        if (e2 != cudaSuccess) return cuda_err(ctx, e2, "end capture");
        e = cudaGraphInstantiate(&G.e, G.g, 0);
        if (e != cudaSuccess) return cuda_err(ctx, e, "graph instantiate");
        // keep at most kMaxGraphs; the oldest entry goes first
        if (ctx->graph_order.size() >= kMaxGraphs) {
            auto old = ctx->graphs.find(ctx->graph_order.front());
            if (old != ctx->graphs.end()) {
                cudaGraphExecDestroy(old->second.second);
                cudaGraphDestroy(old->second.first);
                ctx->graphs.erase(old);
            }
            ctx->graph_order.erase(ctx->graph_order.begin());
        }
        ctx->graphs[keybuf] = std::make_pair(G.g, G.e);
        ctx->graph_order.push_back(keybuf);
        exec = G.e;
        G.g = nullptr; // owned by the context now
        G.e = nullptr;
    }

    int restarts = 0;
    int iters = 0;
    long long launched = 0; // iterations launched: bounds the host loop even if no RHS reports progress
    double worst = 0.0;
    bool converged = false, numeric = false;
    for (;;) {
        // iterate until the device says every RHS stopped, or maxiter
        for (;;) {
            e = cudaGraphLaunch(exec, s);
            if (e != cudaSuccess) return cuda_err(ctx, e, "graph launch");
            launched += chunk;
            st = read_scalars(ctx, S_FLAGS, 1, s);
            if (st) return st;
            const double *f = ctx->h_scal;
            iters = (int)f[F_ITERS];
            if (f[F_NUMERIC] != 0.0) {
                numeric = true;
                break;
            }
            if (f[F_DONE] != 0.0 || iters >= opts->maxiter || launched >= 2LL * opts->maxiter + chunk) break;
        }
        if (numeric) break;
        if (sv.mixed()) {
            // fold the pending low-precision increment into x
            st = blas_accum(ctx, sv.g, rep, kF32, x, sv.x_lo, nullptr, s);
            if (st) return st;
        }
        // true FP64 residual per RHS
        st = sv.true_residual(kFinStore);
        if (st) return st;
        st = read_scalars(ctx, 0, S_NSLOTS, s);
        if (st) return st;
        worst = 0.0;
        int nrhs = sv.g.nrhs;
        for (int r = 0; r < nrhs; ++r) {
            double rr = ctx->h_scal[S_OUT * kMaxRhsSlots + r], bb = ctx->h_scal[S_BB * kMaxRhsSlots + r];
            double rel = bb > 0.0 ? std::sqrt(rr / bb) : 0.0;
            if (!std::isfinite(rel)) numeric = true;
            if (rel > worst || !std::isfinite(rel)) worst = rel;
        }
        if (numeric) break;
        converged = worst <= opts->tol;
        if (converged || iters >= opts->maxiter || restarts >= 20 || launched >= 2LL * opts->maxiter) break;
        // the recurrence stopped early (rounding drift): restart from the true residual
        ++restarts;
        st = sv.true_residual(kFinInit);
        if (!st) st = sv.restart_direction();
        if (st) return st;
    }
    e = cudaEventRecord(ctx->ev1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(ctx->ev1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    if (e != cudaSuccess) return cuda_err(ctx, e, "solve timing");
    st = read_scalars(ctx, S_FLAGS, 1, s);
    if (st) return st;
    if (info) {
        info->iters = iters;
        info->n_reliable_updates = (int)ctx->h_scal[F_NRELIABLE] + restarts;
        info->true_rel_residual = worst;
        info->seconds = ms * 1e-3;
    }
    if (numeric) return set_error(ctx, HR_ERR_NUMERIC, "NaN or Inf in the CG residual");
    if (!converged)
        return set_error(ctx, HR_ERR_NOT_CONVERGED, "not converged: |b-Ax|/|b| = %.3e after %d iterations", worst, iters);
    return HR_OK;
}

} // extern "C"
