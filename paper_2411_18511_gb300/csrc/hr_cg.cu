// hr_cg.cu -- conjugate-gradient solvers on the even-odd normal operator
// A = Mhat^+ Mhat (even sites), the "inverters" of arXiv:2411.18511 Sec. 1
// applied to the even-odd preconditioned operator of Sec. 2.1.
//
// * FP64 CG (Hestenes-Stiefel).  One iteration is four hop launches (the
//   second one reduces |Mhat p|^2 = <p, A p> and sets alpha on the device),
//   one fused x/r update with the |r|^2 reduction (sets beta and the per-RHS
//   convergence flags on the device) and one p update.  No host round trip per
//   iteration.  By default the whole loop is one CUDA graph: a conditional
//   WHILE node whose body is one iteration, its condition set on the device,
//   so a solve is a single graph launch (check_every > 0 instead replays a
//   graph of that many iterations and checks the device flags on the host).
// * Mixed precision with reliable updates (Clark et al., Comput. Phys. Commun.
//   181 (2010) 1517): the recurrence runs on FP32 or FP16 copies of the gauge
//   field and of p, r, q with FP32 arithmetic and an FP32 solution increment.
//   When |r| drops below delta * max|r| since the last update (or below the
//   target), a device-gated block adds the increment into the FP64 solution,
//   recomputes r = b - A x in FP64 and restarts the low-precision residual from
//   it, keeping the search direction.  Convergence is only declared on an FP64
//   residual.  In the one-graph solve the update is a conditional IF node, so
//   iterations without one launch nothing for it.
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

// keep at most kMaxGraphs instantiated graphs in the context; the oldest goes first
void cache_graph(hr_ctx *ctx, const std::string &key, const Graph &G)
{
    if (ctx->graph_order.size() >= kMaxGraphs) {
        auto old = ctx->graphs.find(ctx->graph_order.front());
        if (old != ctx->graphs.end()) {
            cudaGraphExecDestroy(old->second.second);
            cudaGraphDestroy(old->second.first);
            ctx->graphs.erase(old);
        }
        ctx->graph_order.erase(ctx->graph_order.begin());
    }
    ctx->graphs[key] = std::make_pair(G.g, G.e);
    ctx->graph_order.push_back(key);
}

hr_status cuda_err(hr_ctx *ctx, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return HR_OK;
    cudaGetLastError();
    return set_error(ctx, HR_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// The binary16 solver's reliable updates use the FP32 tier while |r| stays above
// kDeltaMid times the last FP64 residual: r_ref - A_32 x_mid carries an error of
// about 1e-7 |r_ref| (FP32 links and arithmetic), 0.1 % of |r| at the switch.
constexpr double kDeltaMid = 1e-4;

hr_status init_scalars(hr_ctx *ctx, int nrhs, double tol, double delta, int maxiter, cudaStream_t s,
                       double delta_mid = 0.0)
{
    std::vector<double> h(kScalDoubles, 0.0);
    for (int r = 0; r < nrhs; ++r) h[S_ACTIVE * kMaxRhsSlots + r] = 1.0;
    h[S_DELTA2 * kMaxRhsSlots + 0] = delta * delta;
    h[S_DELTA2 * kMaxRhsSlots + 1] = tol * tol;
    h[S_DELTA2 * kMaxRhsSlots + 2] = maxiter;
    h[S_DELTA2 * kMaxRhsSlots + 3] = delta_mid * delta_mid;
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

enum CtlWhat { kCtlGate = 0, kCtlLoop = 1 };
constexpr int kIterPerPass = 8; // iterations per pass of the device loop body

// Device-side control of the solve graph.  kCtlGate: run the reliable update
// (IF node) this iteration?  kCtlLoop: run another pass of the loop body (WHILE
// node)?  The loop stops when the done flag is up (every RHS stopped, maxiter
// reached or a NaN seen) and, as a backstop, after 2 maxiter + 64 passes.
__global__ void k_cg_ctl(double *scal, cudaGraphConditionalHandle h, int what, int maxiter)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double *f = scal + S_FLAGS * kMaxRhsSlots;
    const bool done = f[F_DONE] != 0.0;
    unsigned v;
    if (what == kCtlGate) {
        v = (!done && f[F_GATE] != 0.0) ? 1u : 0u;
    } else {
        f[F_BODY] += 1.0;
        v = (!done && f[F_ITERS] < (double)maxiter && f[F_BODY] < 2.0 * maxiter + 64.0) ? 1u : 0u;
    }
    cudaGraphSetConditional(h, v);
}

struct Solver {
    hr_ctx *ctx;
    Geom g;
    double m0;
    int rep;
    hr_solver_opts o;
    const void *gauge;
    const void *clov64;  // packed FP64 clover field, or nullptr (Wilson)
    const void *b;
    void *x;
    cudaStream_t s;
    const void *b_user; // the caller's source; b is its scaled copy bs64 once start() ran
    // FP64 buffers
    void *r64, *p64, *q64, *u64, *t64, *bs64;
    // low precision buffers
    void *gauge_lo, *r_lo, *p_lo, *q_lo, *u_lo, *t_lo, *x_lo;
    void *clov_lo; // FP32 copy of the clover field (mixed solvers)
    // the FP32 tier of the binary16 solver's reliable updates: the FP32 gauge,
    // the correction since the last FP64 residual, and the FP32 operator's vectors
    void *gauge_mid, *x_mid, *q_mid, *t_mid, *u_mid;
    size_t h64, hlo, h32, glo;

    bool mixed() const { return o.inner_prec != HR_F64; }
    // binary16 inner solves refresh their residual in FP32 between FP64 ones
    bool two_tier() const { return o.inner_prec == HR_F16; }

    static size_t layout(const Geom &g, int rep, const hr_solver_opts &o, bool clover, Solver *sv, void *work)
    {
        size_t h64 = spinor_half_bytes(g, rep, kF64);
        char *w = (char *)work;
        size_t off = 0;
        auto take = [&](size_t n) -> void * {
            void *p = w ? (void *)(w + off) : nullptr;
            off += (n + 255) & ~(size_t)255;
            return p;
        };
        void *bs = take(h64);
        if (sv) sv->bs64 = bs;
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
            void *cl = clover ? take(4 * clover_half_bytes(g, rep, kF32)) : nullptr;
            void *gm = nullptr, *xm = nullptr, *qm = nullptr, *tm = nullptr, *um = nullptr;
            if (o.inner_prec == HR_F16) {
                gm = take(gauge_bytes(g, rep, kF32));
                xm = take(h32); qm = take(h32); tm = take(h32); um = take(h32);
            }
            if (sv) {
                sv->gauge_mid = gm; sv->x_mid = xm; sv->q_mid = qm; sv->t_mid = tm; sv->u_mid = um;
                sv->clov_lo = cl;
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
        return apply_eo_op(ctx, g, m0, rep, kF64, HR_OP_NORMAL, gauge, v, ax, t64, u64, fin, gate, done, s, nullptr,
                           clov64);
    }

    // One iteration = part_a (q = A p with <p,q> -> alpha; x, r update with
    // |r|^2 -> beta), then for the mixed solver the reliable update, then
    // part_b (p = r + beta p).
    hr_status part_a()
    {
        const double *done = flag_ptr(ctx, F_DONE);
        if (!mixed()) {
            // q = A p with the x/r update and |r|^2 fused into the last hop
            const CgFuse fz{x, p64, r64, kFinBeta};
            return apply_eo_op(ctx, g, m0, rep, kF64, HR_OP_NORMAL, gauge, p64, q64, t64, u64, kFinAlpha, nullptr,
                               done, s, &fz, clov64);
        }
        // p, r in the inner precision, x_lo in FP32: fused as above (the
        // last hop's epilogue updates x_lo and r from q in registers)
        const CgFuse fz{x_lo, p_lo, r_lo, kFinBetaMixed};
        return apply_eo_op(ctx, g, m0, rep, o.inner_prec, HR_OP_NORMAL, gauge_lo, p_lo, q_lo, t_lo, u_lo, kFinAlpha,
                           nullptr, done, s, &fz, clov_lo);
    }

    // x += x_lo, r = b - A x in FP64, restart the low-precision residual;
    // every launch skips its work unless *gate != 0 (gate == nullptr: always run)
    //
    // Two tiers for the binary16 solver (the gate of the open tier set on the
    // device by the recurrence's last reduction; gate is then unused):
    //   FP32: x_mid += x_lo, r_lo = r_ref - A_32 x_mid, with r_ref the last FP64
    //         residual (r64): accurate to FP32 relative to r_ref, which is all a
    //         binary16 recurrence can use while |r| > delta_mid |r_ref|;
    //   FP64: x += x_lo + x_mid, r = b - A x (the reference and the stop test).
    hr_status reliable_update(const double *gate)
    {
        if (two_tier()) {
            const double *g1 = flag_ptr(ctx, F_TIER1), *g2 = flag_ptr(ctx, F_TIER2);
            hr_status st = blas_accum(ctx, g, rep, kF32, x_mid, x_lo, g1, s, kF32);
            if (!st)
                st = apply_eo_op(ctx, g, m0, rep, kF32, HR_OP_NORMAL, gauge_mid, x_mid, q_mid, t_mid, u_mid, kFinNone,
                                 g1, nullptr, s, nullptr, clov_lo);
            if (!st) st = blas_residual(ctx, g, rep, r64, q_mid, nullptr, kFinMid, g1, kF16, r_lo, s, kF32);
            if (!st) st = blas_accum(ctx, g, rep, kF32, x, x_lo, g2, s);
            if (!st) st = blas_accum(ctx, g, rep, kF32, x, x_mid, g2, s);
            if (!st) st = apply64(x, q64, kFinNone, g2, nullptr);
            if (!st) st = blas_residual(ctx, g, rep, b, q64, r64, kFinResidual, g2, o.inner_prec, r_lo, s);
            return st;
        }
        hr_status st = blas_accum(ctx, g, rep, kF32, x, x_lo, gate, s);
        if (!st) st = apply64(x, q64, kFinNone, gate, nullptr);
        if (!st) st = blas_residual(ctx, g, rep, b, q64, r64, kFinResidual, gate, o.inner_prec, r_lo, s);
        return st;
    }

    hr_status part_b()
    {
        if (!mixed()) return blas_p(ctx, g, rep, kF64, kF64, p64, r64, s);
        return blas_p(ctx, g, rep, o.inner_prec, o.inner_prec, p_lo, r_lo, s);
    }

    // the iteration with the reliable update gated inside its kernels
    hr_status iteration()
    {
        hr_status st = part_a();
        if (!st && mixed()) st = reliable_update(flag_ptr(ctx, F_GATE));
        if (!st) st = part_b();
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

    // Rescale the source by a power of two per right-hand side (exact) so that
    // its largest component lies in [0.5, 1): the vectors the recurrence
    // iterates then stay far from both ends of the float exponent range that
    // the double-float pairs keep, whatever the scale of the caller's b.  x
    // is solved for in the same units (a guess is scaled along) and scaled
    // back by finish().
    hr_status scale_source()
    {
        hr_status st = blas_source_scale(ctx, g, rep, b_user, s);
        if (st) return st;
        st = read_scalars(ctx, S_FLAGS, 1, s);
        if (st) return st;
        if (ctx->h_scal[F_RANGE] != 0.0)
            return set_error(ctx, HR_ERR_UNSUPPORTED,
                             "the source's largest component is below 2^-100 = 7.9e-31: its FP64 pairs have lost low "
                             "bits (scale b up)");
        st = blas_scale(ctx, g, rep, b_user, bs64, 0, s);
        if (!st && o.x0_is_guess) st = blas_scale(ctx, g, rep, x, x, 0, s);
        b = bs64;
        return st;
    }

    // x back in the caller's units
    hr_status finish() { return blas_scale(ctx, g, rep, x, x, 1, s); }

    hr_status start()
    {
        hr_status st = init_scalars(ctx, g.nrhs, o.tol, o.reliable_delta, o.maxiter, s, two_tier() ? kDeltaMid : 0.0);
        if (st) return st;
        st = scale_source();
        if (st) return st;
        if (mixed()) {
            st = gauge_convert(ctx, make_geom_gauge(), rep, o.inner_prec, gauge, gauge_lo, s);
            if (!st && clov64) st = clover_convert_f32(ctx, g, rep, clov64, clov_lo, s);
            if (!st && two_tier()) st = gauge_convert(ctx, make_geom_gauge(), rep, kF32, gauge, gauge_mid, s);
            if (!st && two_tier()) st = blas_zero(ctx, g, rep, kF32, x_mid, s);
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

// The whole solve loop as one graph: a WHILE node whose body is `per_pass`
// iterations, with the reliable update of the mixed solver in an IF node per
// iteration.  Kernels set every condition on the device (k_cg_ctl), so a solve
// is one graph launch.  A pass of a WHILE body and a taken IF node each cost
// about 25 us of scheduling on this hardware (a skipped IF about 9 us), so the
// body holds several iterations; those after convergence skip their work on
// the done flag.
hr_status capture_while_graph(Solver &sv, int per_pass, cudaGraph_t *out)
{
    hr_ctx *ctx = sv.ctx;
    const cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
    cudaGraph_t G = nullptr;
    cudaStream_t cs = nullptr;
    cudaStream_t user = sv.s;
    bool capturing = false;
    hr_status st = HR_OK;
    cudaError_t e = cudaSuccess;
    auto fail = [&](const char *what) -> hr_status {
        if (capturing) {
            cudaGraph_t junk = nullptr;
            cudaStreamEndCapture(cs, &junk);
        }
        if (cs) cudaStreamDestroy(cs);
        if (G) cudaGraphDestroy(G);
        sv.s = user;
        if (st) return st;
        return cuda_err(ctx, e != cudaSuccess ? e : cudaErrorUnknown, what);
    };
    auto begin = [&](cudaGraph_t into, const cudaGraphNode_t *dep, size_t ndep) {
        e = cudaStreamBeginCaptureToGraph(cs, into, dep, nullptr, ndep, mode);
        capturing = e == cudaSuccess;
        return capturing;
    };
    auto end = [&]() {
        cudaGraph_t same = nullptr;
        capturing = false;
        e = cudaStreamEndCapture(cs, &same);
        return e == cudaSuccess;
    };
    auto cond_node = [&](cudaGraph_t parent, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                         const cudaGraphNode_t *dep, size_t ndep, cudaGraphNode_t *node, cudaGraph_t *child) {
        cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
        np.conditional.handle = h;
        np.conditional.type = type;
        np.conditional.size = 1;
        e = cudaGraphAddNode(node, parent, dep, nullptr, ndep, &np);
        if (e == cudaSuccess) *child = np.conditional.phGraph_out[0];
        return e == cudaSuccess;
    };
    const int maxiter = sv.o.maxiter;

    if ((e = cudaGraphCreate(&G, 0)) != cudaSuccess) return fail("graph create");
    if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) return fail("capture stream");
    cudaGraphConditionalHandle hloop;
    if ((e = cudaGraphConditionalHandleCreate(&hloop, G, 1, cudaGraphCondAssignDefault)) != cudaSuccess)
        return fail("loop condition");
    cudaGraphNode_t wnode;
    cudaGraph_t body = nullptr;
    if (!cond_node(G, hloop, cudaGraphCondTypeWhile, nullptr, 0, &wnode, &body)) return fail("while node");
    sv.s = cs;
    if (!begin(body, nullptr, 0)) return fail("begin capture");
    for (int k = 0; k < per_pass; ++k) {
        if ((st = sv.part_a())) return fail("iteration");
        if (sv.mixed()) {
            // each IF node has its own condition handle
            cudaGraphConditionalHandle hgate;
            if ((e = cudaGraphConditionalHandleCreate(&hgate, body, 0, cudaGraphCondAssignDefault)) != cudaSuccess)
                return fail("gate condition");
            k_cg_ctl<<<1, 32, 0, cs>>>(ctx->d_scal, hgate, kCtlGate, maxiter);
            if ((st = check_launch(ctx, "cg control"))) return fail("cg control");
            cudaStreamCaptureStatus cst;
            const cudaGraphNode_t *d = nullptr;
            size_t nd = 0;
            if ((e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &d, nullptr, &nd)) != cudaSuccess)
                return fail("capture info");
            std::vector<cudaGraphNode_t> deps(d, d + nd);
            if (!end()) return fail("end capture");
            cudaGraphNode_t inode;
            cudaGraph_t ifbody = nullptr;
            if (!cond_node(body, hgate, cudaGraphCondTypeIf, deps.data(), deps.size(), &inode, &ifbody))
                return fail("if node");
            if (!begin(ifbody, nullptr, 0)) return fail("begin capture");
            if ((st = sv.reliable_update(nullptr))) return fail("reliable update");
            if (!end()) return fail("end capture");
            if (!begin(body, &inode, 1)) return fail("begin capture");
        }
        if ((st = sv.part_b())) return fail("iteration");
    }
    k_cg_ctl<<<1, 32, 0, cs>>>(ctx->d_scal, hloop, kCtlLoop, maxiter);
    if ((st = check_launch(ctx, "cg control"))) return fail("cg control");
    if (!end()) return fail("end capture");
    cudaStreamDestroy(cs);
    sv.s = user;
    *out = G;
    return HR_OK;
}

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

} // extern "C"

namespace {

size_t cg_workspace(hr_lattice lat, hr_rep rep, const hr_solver_opts *opts, bool clover)
{
    if (!opts || !valid_rep(rep) || !valid_prec(opts->inner_prec) || opts->n_rhs < 1 || opts->n_rhs > kMaxRhs)
        return 0;
    if (hr_spinor_packed_bytes(lat, rep, HR_F64, HR_EVEN, opts->n_rhs) == 0) return 0;
    return Solver::layout(make_geom(lat, opts->n_rhs), rep, *opts, clover, nullptr, nullptr);
}

// the CG of hr_cg_solve and hr_cg_solve_clover (clover == nullptr: Wilson, m0 used)
hr_status cg_solve(hr_ctx *ctx, hr_lattice lat, double m0, hr_rep rep, const hr_solver_opts *opts, const void *gauge,
                   const void *clover, const void *b, void *x, hr_solve_info *info, void *work, size_t work_bytes,
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
    st = check_buffers(ctx, {gauge, b, x}, {}, {work, clover});
    if (st) return st;
    if (b == x) return set_error(ctx, HR_ERR_INVALID_ARG, "b and x must not alias");
    if (!clover && !(4.0 + m0 != 0.0)) return set_error(ctx, HR_ERR_INVALID_ARG, "4 + m0 must be nonzero");
    size_t need = cg_workspace(lat, rep, opts, clover != nullptr);
    if (!work || work_bytes < need)
        return set_error(ctx, HR_ERR_WORKSPACE, "workspace of %zu bytes needed, %zu given", need, work_bytes);

    // values packed out of range since the last check (this synchronises the stream)
    st = consume_pack_status(ctx, (cudaStream_t)stream);
    if (st) return st;

    Solver sv{};
    sv.ctx = ctx;
    sv.g = make_geom(lat, opts->n_rhs);
    sv.m0 = m0;
    sv.rep = rep;
    sv.o = *opts;
    sv.gauge = gauge;
    sv.clov64 = clover;
    sv.b_user = b;
    sv.b = b;
    sv.x = x;
    sv.s = (cudaStream_t)stream;
    Solver::layout(sv.g, rep, *opts, clover != nullptr, &sv, work);
    cudaStream_t s = sv.s;

    cudaError_t e = cudaEventRecord(ctx->ev0, s);
    if (e != cudaSuccess) return cuda_err(ctx, e, "event record");
    st = sv.start();
    if (st) return st;

    // check_every == 0: the whole loop is one graph (device-side WHILE);
    // check_every == N: a graph of N iterations, replayed with a host check after each
    const bool device_loop = opts->check_every <= 0;
    int chunk = device_loop ? kIterPerPass : opts->check_every;
    if (chunk > opts->maxiter) chunk = opts->maxiter;
    // The graph bakes in every launch parameter: buffers, lattice, m0, maxiter,
    // the hop shapes in use.  Solves that repeat them (a benchmark, an MD trajectory
    // with persistent buffers) reuse the instantiated graph from the context.
    char keybuf[512];
    {
        HopChoice c64 = hop_choice(ctx, sv.g, rep, kF64), clo = hop_choice(ctx, sv.g, rep, opts->inner_prec);
        // the reducing launches' shapes are baked in too
        const HopChoice f64 = hop_choice_fin(ctx, sv.g, rep, kF64), flo = hop_choice_fin(ctx, sv.g, rep, opts->inner_prec),
                        f32 = hop_choice_fin(ctx, sv.g, rep, kF32), c32 = hop_choice(ctx, sv.g, rep, kF32);
        unsigned long long m0bits;
        std::memcpy(&m0bits, &m0, sizeof m0bits);
        // the twist angles select the kernel and its phases
        unsigned long long tb[4];
        std::memcpy(tb, lat.theta, sizeof tb);
        snprintf(keybuf, sizeof keybuf,
                 "cg:%d:%d:%d:%d:%d:%d:%d:%llx:%d:%d:%d:%p:%p:%p:%p:%p:%d.%d:%d.%d:%d.%d:%d.%d:%d.%d:%d.%d:%zu:"
                 "%llx.%llx.%llx.%llx",
                 lat.dims[0], lat.dims[1], lat.dims[2], lat.dims[3], sv.g.nrhs, rep, opts->inner_prec, m0bits,
                 device_loop ? -chunk : chunk,
                 opts->maxiter, (int)sizeof(void *), gauge, clover, b, x, work, c64.variant, c64.block, clo.variant,
                 clo.block, f64.variant, f64.block, flo.variant, flo.block, c32.variant, c32.block, f32.variant,
                 f32.block, work_bytes, tb[0], tb[1], tb[2], tb[3]);
    }
    cudaGraphExec_t exec = nullptr;
    auto cached = ctx->graphs.find(keybuf);
    if (cached != ctx->graphs.end()) {
        exec = cached->second.second;
    } else if (device_loop) {
        Graph G;
        st = capture_while_graph(sv, chunk, &G.g);
        if (st) return st;
        e = cudaGraphInstantiate(&G.e, G.g, 0);
        if (e != cudaSuccess) return cuda_err(ctx, e, "graph instantiate");
        cache_graph(ctx, keybuf, G);
        exec = G.e;
        G.g = nullptr; // owned by the context now
        G.e = nullptr;
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
        cache_graph(ctx, keybuf, G);
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
            launched += device_loop ? 1 : chunk;
            st = read_scalars(ctx, S_FLAGS, 1, s);
            if (st) return st;
            const double *f = ctx->h_scal;
            iters = (int)f[F_ITERS];
            if (f[F_NUMERIC] != 0.0) {
                numeric = true;
                break;
            }
            if (device_loop || f[F_DONE] != 0.0 || iters >= opts->maxiter || launched >= 2LL * opts->maxiter + chunk)
                break;
        }
        if (numeric) break;
        // A mixed solve normally stops inside a reliable update: the recurrence's
        // convergence opens the gate, and only the FP64 residual it recomputes
        // stops a right-hand side.  Its x_lo is then folded into x and S_OUT
        // holds |b - A x|^2 for the x being returned, so the same residual is
        // not computed twice.  Otherwise (maxiter, the FP64 solver) compute it.
        const bool have_true = sv.mixed() && ctx->h_scal[F_TRUERES] != 0.0;
        if (!have_true) {
            if (sv.mixed()) {
                // fold the pending low-precision increments into x
                st = blas_accum(ctx, sv.g, rep, kF32, x, sv.x_lo, nullptr, s);
                if (!st && sv.two_tier()) st = blas_accum(ctx, sv.g, rep, kF32, x, sv.x_mid, nullptr, s);
                if (st) return st;
            }
            // true FP64 residual per RHS
            st = sv.true_residual(kFinStore);
            if (st) return st;
        }
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
    st = sv.finish();
    if (st) return st;
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
    if (ctx->h_scal[F_DEVERR] != 0.0)
        return set_error(ctx, HR_ERR_TIMEOUT, "a bulk copy into shared memory did not land within its time limit");
    if (numeric) return set_error(ctx, HR_ERR_NUMERIC, "NaN or Inf in the CG residual");
    if (!converged)
        return set_error(ctx, HR_ERR_NOT_CONVERGED, "not converged: |b-Ax|/|b| = %.3e after %d iterations", worst, iters);
    return HR_OK;
}

} // namespace

extern "C" {

size_t hr_cg_workspace_bytes(hr_lattice lat, hr_rep rep, const hr_solver_opts *opts)
{
    return cg_workspace(lat, rep, opts, false);
}

size_t hr_cg_clover_workspace_bytes(hr_lattice lat, hr_rep rep, const hr_solver_opts *opts)
{
    return cg_workspace(lat, rep, opts, true);
}

hr_status hr_cg_solve(hr_ctx *ctx, hr_lattice lat, double m0, hr_rep rep, const hr_solver_opts *opts,
                      const void *gauge, const void *b, void *x, hr_solve_info *info, void *work, size_t work_bytes,
                      hr_stream stream)
{
    return cg_solve(ctx, lat, m0, rep, opts, gauge, nullptr, b, x, info, work, work_bytes, stream);
}

hr_status hr_cg_solve_clover(hr_ctx *ctx, hr_lattice lat, hr_rep rep, const hr_solver_opts *opts, const void *gauge,
                             const void *clover, const void *b, void *x, hr_solve_info *info, void *work,
                             size_t work_bytes, hr_stream stream)
{
    if (!ctx) return HR_ERR_INVALID_ARG;
    if (info) std::memset(info, 0, sizeof *info);
    if (!clover) return set_error(ctx, HR_ERR_INVALID_ARG, "null clover field");
    return cg_solve(ctx, lat, 0.0, rep, opts, gauge, clover, b, x, info, work, work_bytes, stream);
}

} // extern "C"
