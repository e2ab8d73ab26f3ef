// hr_solve.cu -- full-lattice solves through the even-odd preconditioned
// operator (arXiv:2411.18511 Sec. 2.1: the Schur form "used mainly in the HMC").
//
// D x = b on all sites, with D = A - 1/2 H and A = 4 + m0, reduces to the even
// sites:
//   source       bhat = b_e - D_eo b_o / A  = b_e + H_eo b_o / (2A)
//   Schur system Mhat x_e = bhat, solved as Mhat^+ Mhat x_e = Mhat^+ bhat (CG)
//   reconstruct  x_o = (b_o - D_oe x_e) / A = b_o / A + H_oe x_e / (2A)
// D^+ D x = b is two such solves: D^+ = g5 D g5 gives x = D^-1 g5 D^-1 g5 b.
// Every step runs in the library's kernels (one fused hop launch each for the
// source and the reconstruction, the CG solver for the Schur system).
#include <cmath>
#include <cstring>

#include "hr_host.h"

using namespace hr;

namespace {

struct FullWork {
    void *cg;     // hr_cg_solve workspace
    void *bhat;   // even half
    void *rhs;    // even half: Mhat^+ bhat
    void *t1, *t2; // full fields (t2: D^+ D only)
    size_t cg_bytes;
};

size_t layout_full(hr_lattice lat, hr_rep rep, const hr_solver_opts *o, int system, bool clover, char *w,
                   FullWork *fw)
{
    const size_t half = hr_spinor_packed_bytes(lat, rep, HR_F64, HR_EVEN, 1);
    const size_t cgb = clover ? hr_cg_clover_workspace_bytes(lat, rep, o) : hr_cg_workspace_bytes(lat, rep, o);
    size_t off = 0;
    auto take = [&](size_t n) -> void * {
        void *p = w ? (void *)(w + off) : nullptr;
        off += (n + 255) & ~(size_t)255;
        return p;
    };
    void *cg = take(cgb), *bhat = take(half), *rhs = take(half);
    void *t1 = take(2 * half), *t2 = nullptr; // t1: residual (and D^+ D's g5 b)
    if (system == HR_SYSTEM_DDAG_D) t2 = take(2 * half);
    if (fw) *fw = FullWork{cg, bhat, rhs, t1, t2, cgb};
    return off;
}

// out (parity p) = alpha aux + beta H in (one hop launch with its fused
// epilogue); with a clover half-field, out = A (alpha aux + beta H in)
hr_status hop_axpy(hr_ctx *ctx, const Geom &g, int rep, int p, const void *gauge, const void *in, const void *aux,
                   void *out, double alpha, double beta, cudaStream_t s, const void *clov_out = nullptr)
{
    HopLaunch L{};
    L.p = p;
    L.gauge = gauge;
    L.in = in;
    L.aux = aux;
    L.out = out;
    L.alpha = alpha;
    L.beta = beta;
    L.clov = clov_out;
    L.clov_mode = clov_out ? kClovOut : kClovNone;
    return launch_hop(ctx, g, rep, kF64, L, s);
}

// x = D^-1 b (full packed FP64 fields), through the Schur system; with a
// clover field (FP64) the diagonal is A instead of 4 + m0
hr_status solve_d(hr_ctx *ctx, hr_lattice lat, double m0, int rep, const hr_solver_opts *o, const void *gauge,
                  const void *clover, const void *b, void *x, const FullWork &w, hr_solve_info *info, cudaStream_t s)
{
    const Geom g = make_geom(lat, 1);
    const size_t half = spinor_half_bytes(g, rep, kF64);
    const char *b_e = (const char *)b, *b_o = b_e + half;
    char *x_e = (char *)x, *x_o = x_e + half;
    hr_status st;
    if (clover) {
        // bhat = b_e + H_eo (A_oo^-1 b_o) / 2, A_oo^-1 b_o in x_o
        const void *inv_odd = clover_half(clover, g, rep, kF64, true, 1);
        st = clover_apply_half(ctx, g, rep, kF64, inv_odd, b_o, x_o, s);
        if (!st) st = hop_axpy(ctx, g, rep, 0, gauge, x_o, b_e, w.bhat, 1.0, 0.5, s);
    } else {
        // bhat = b_e + H_eo b_o / (2A)
        st = hop_axpy(ctx, g, rep, 0, gauge, b_o, b_e, w.bhat, 1.0, 0.5 / (4.0 + m0), s);
    }
    // rhs = Mhat^+ bhat (x_o serves as the odd temporary)
    if (!st)
        st = apply_eo_op(ctx, g, m0, rep, kF64, HR_OP_SCHUR_DAG, gauge, w.bhat, w.rhs, x_o, nullptr, kFinNone,
                         nullptr, nullptr, s, nullptr, clover);
    if (st) return st;
    // Mhat^+ Mhat x_e = rhs
    hr_solver_opts oo = *o;
    oo.n_rhs = 1;
    oo.x0_is_guess = 0;
    if (clover)
        st = hr_cg_solve_clover(ctx, lat, (hr_rep)rep, &oo, gauge, clover, w.rhs, x_e, info, w.cg, w.cg_bytes,
                                (hr_stream)s);
    else
        st = hr_cg_solve(ctx, lat, m0, (hr_rep)rep, &oo, gauge, w.rhs, x_e, info, w.cg, w.cg_bytes, (hr_stream)s);
    if (st) return st;
    if (clover) // x_o = A_oo^-1 (b_o + H_oe x_e / 2)
        return hop_axpy(ctx, g, rep, 1, gauge, x_e, b_o, x_o, 1.0, 0.5, s, clover_half(clover, g, rep, kF64, true, 1));
    // x_o = b_o / A + H_oe x_e / (2A)
    const double A = 4.0 + m0;
    return hop_axpy(ctx, g, rep, 1, gauge, x_e, b_o, x_o, 1.0 / A, 0.5 / A, s);
}

hr_status gamma5_full(hr_ctx *ctx, const Geom &g, int rep, void *v, cudaStream_t s)
{
    const size_t half = spinor_half_bytes(g, rep, kF64);
    hr_status st = blas_gamma5(ctx, g, rep, v, s);
    if (!st) st = blas_gamma5(ctx, g, rep, (char *)v + half, s);
    return st;
}

// |v|^2 over both halves of a full field, on the host
hr_status norm2_full(hr_ctx *ctx, const Geom &g, int rep, const void *v, double &out, cudaStream_t s)
{
    const size_t half = spinor_half_bytes(g, rep, kF64);
    double sum = 0.0;
    for (int h = 0; h < 2; ++h) {
        hr_status st = blas_norm2(ctx, g, rep, kF64, (const char *)v + h * half, kFinStore, s);
        if (st) return st;
        cudaError_t e = cudaMemcpyAsync(ctx->h_scal, ctx->d_scal + S_OUT * kMaxRhsSlots, sizeof(double),
                                        cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return set_error(ctx, HR_ERR_CUDA, "norm readback: %s", cudaGetErrorString(e));
        sum += ctx->h_scal[0];
    }
    out = sum;
    return HR_OK;
}


size_t full_workspace(hr_lattice lat, hr_rep rep, const hr_solver_opts *opts, hr_system system, bool clover)
{
    if (!opts || (system != HR_SYSTEM_D && system != HR_SYSTEM_DDAG_D)) return 0;
    if (opts->n_rhs != 1 || opts->inner_prec < HR_F64 || opts->inner_prec > HR_F16) return 0;
    if (!valid_rep(rep) || hr_spinor_packed_bytes(lat, rep, HR_F64, HR_EVEN, 1) == 0) return 0;
    if (hr_cg_workspace_bytes(lat, rep, opts) == 0) return 0;
    return layout_full(lat, rep, opts, system, clover, nullptr, nullptr);
}

// hr_solve_full and hr_solve_full_clover (clover == nullptr: Wilson with m0)
hr_status solve_full(hr_ctx *ctx, hr_lattice lat, double m0, hr_rep rep, const hr_solver_opts *opts, hr_system system,
                     const void *gauge, const void *clover, const void *b, void *x, hr_solve_info *info, void *work,
                     size_t work_bytes, hr_stream stream)
{
    if (!ctx) return HR_ERR_INVALID_ARG;
    if (info) std::memset(info, 0, sizeof *info);
    if (!opts) return set_error(ctx, HR_ERR_INVALID_ARG, "null options");
    if (system != HR_SYSTEM_D && system != HR_SYSTEM_DDAG_D) return set_error(ctx, HR_ERR_INVALID_ARG, "bad system");
    if (opts->n_rhs != 1) return set_error(ctx, HR_ERR_UNSUPPORTED, "full-lattice solve: one right-hand side");
    if (!valid_rep(rep)) return set_error(ctx, HR_ERR_INVALID_ARG, "bad rep");
    hr_status st = validate_lattice(ctx, lat, 1);
    if (st) return st;
    st = check_buffers(ctx, {gauge, b, x}, {}, {work, clover});
    if (st) return st;
    if (b == x) return set_error(ctx, HR_ERR_INVALID_ARG, "b and x must not alias");
    if (!clover && !(4.0 + m0 != 0.0)) return set_error(ctx, HR_ERR_INVALID_ARG, "4 + m0 must be nonzero");
    const size_t need = full_workspace(lat, rep, opts, system, clover != nullptr);
    if (need == 0) return set_error(ctx, HR_ERR_INVALID_ARG, "bad solver options");
    if (!work || work_bytes < need)
        return set_error(ctx, HR_ERR_WORKSPACE, "workspace of %zu bytes needed, %zu given", need, work_bytes);
    FullWork w;
    layout_full(lat, rep, opts, system, clover != nullptr, (char *)work, &w);
    cudaStream_t s = (cudaStream_t)stream;
    const Geom g = make_geom(lat, 1);
    const size_t full = 2 * spinor_half_bytes(g, rep, kF64);

    hr_solve_info i1{}, i2{};
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    cudaEventRecord(t0, s);
    if (system == HR_SYSTEM_D) {
        st = solve_d(ctx, lat, m0, rep, opts, gauge, clover, b, x, w, &i1, s);
    } else {
        // x = D^-1 g5 D^-1 g5 b
        cudaError_t e = cudaMemcpyAsync(w.t1, b, full, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) st = set_error(ctx, HR_ERR_CUDA, "copy: %s", cudaGetErrorString(e));
        if (!st) st = gamma5_full(ctx, g, rep, w.t1, s);
        if (!st) st = solve_d(ctx, lat, m0, rep, opts, gauge, clover, w.t1, w.t2, w, &i1, s);
        if (!st) st = gamma5_full(ctx, g, rep, w.t2, s);
        if (!st) st = solve_d(ctx, lat, m0, rep, opts, gauge, clover, w.t2, x, w, &i2, s);
    }
    cudaEventRecord(t1, s);
    float ms = 0.f;
    if (cudaEventSynchronize(t1) == cudaSuccess) cudaEventElapsedTime(&ms, t0, t1);
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (st) return st;

    // the true relative residual of the full system, recomputed in FP64:
    // r = D x - b (or D^+ D x - b = g5 D g5 D x - b) in t1
    void *r = w.t1;
    auto dirac = [&](const void *in, void *out) {
        return clover ? hr_dirac_apply_clover(ctx, lat, rep, HR_F64, gauge, clover, in, out, stream)
                      : hr_dirac_apply(ctx, lat, m0, rep, HR_F64, gauge, in, out, stream);
    };
    if (system == HR_SYSTEM_D) {
        st = dirac(x, r);
    } else {
        st = dirac(x, w.t2);
        if (!st) st = gamma5_full(ctx, g, rep, w.t2, s);
        if (!st) st = dirac(w.t2, r);
        if (!st) st = gamma5_full(ctx, g, rep, r, s);
    }
    const size_t half = spinor_half_bytes(g, rep, kF64);
    for (int h = 0; h < 2 && !st; ++h)
        st = blas_axpy(ctx, g, rep, -1.0, (const char *)b + h * half, (char *)r + h * half, s);
    double rr = 0.0, bb = 0.0;
    if (!st) st = norm2_full(ctx, g, rep, r, rr, s);
    if (!st) st = norm2_full(ctx, g, rep, b, bb, s);
    if (st) return st;
    const double rel = bb > 0.0 ? std::sqrt(rr / bb) : 0.0;
    if (info) {
        info->iters = i1.iters + i2.iters;
        info->n_reliable_updates = i1.n_reliable_updates + i2.n_reliable_updates;
        info->true_rel_residual = rel;
        info->seconds = ms * 1e-3;
    }
    if (!std::isfinite(rel)) return set_error(ctx, HR_ERR_NUMERIC, "NaN or Inf in the full-system residual");
    return HR_OK;
}

} // namespace

extern "C" {

size_t hr_solve_full_workspace_bytes(hr_lattice lat, hr_rep rep, const hr_solver_opts *opts, hr_system system)
{
    return full_workspace(lat, rep, opts, system, false);
}

size_t hr_solve_full_clover_workspace_bytes(hr_lattice lat, hr_rep rep, const hr_solver_opts *opts, hr_system system)
{
    return full_workspace(lat, rep, opts, system, true);
}

hr_status hr_solve_full(hr_ctx *ctx, hr_lattice lat, double m0, hr_rep rep, const hr_solver_opts *opts,
                        hr_system system, const void *gauge, const void *b, void *x, hr_solve_info *info, void *work,
                        size_t work_bytes, hr_stream stream)
{
    return solve_full(ctx, lat, m0, rep, opts, system, gauge, nullptr, b, x, info, work, work_bytes, stream);
}

hr_status hr_solve_full_clover(hr_ctx *ctx, hr_lattice lat, hr_rep rep, const hr_solver_opts *opts, hr_system system,
                               const void *gauge, const void *clover, const void *b, void *x, hr_solve_info *info,
                               void *work, size_t work_bytes, hr_stream stream)
{
    if (!ctx) return HR_ERR_INVALID_ARG;
    if (info) std::memset(info, 0, sizeof *info);
    if (!clover) return set_error(ctx, HR_ERR_INVALID_ARG, "null clover field");
    return solve_full(ctx, lat, 0.0, rep, opts, system, gauge, clover, b, x, info, work, work_bytes, stream);
}

} // extern "C"
