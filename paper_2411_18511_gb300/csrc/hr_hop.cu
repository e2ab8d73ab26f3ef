// hr_hop.cu -- the even-odd Wilson hopping kernel and the operators built on it:
// D_eo / D_oe, the Schur complement Mhat, Mhat^+, Mhat^+ Mhat and the full D.
//
// One thread per output (virtual) site.  For each of the 8 directions the
// thread takes the neighbour spinor (16-byte vectors, AoSoA blocks of 32
// sites), projects it to a half spinor with (1 -/+ g_mu), multiplies both spin
// components by the link rebuilt in registers from its quaternion (or by the
// stored 3x3 adjoint matrix), and adds the two rebuilt spin pairs into the
// accumulator.  The periodic wrap is resolved in the neighbour index; there is
// no halo.  The epilogue forms out = alpha*aux + beta*[g5] H [g5] in and, when
// asked, reduces |out|^2 per right-hand side (fused CG reduction).
//
// This file holds the plain unrolled kernels (variants 0 and 7), the dispatch
// over all variants (the other families are in hr_hop_staged.cu, hr_hop_loop.cu,
// hr_hop_tile.cu, hr_hop_x2.cu, hr_hop_half.cu, hr_hop_p2.cu and hr_hop_chunk.cu;
// hr_hop_fam.h lists them; lattices with
// twisted boundaries take the kernel of hr_hop_twist.cu), the operators built
// from hops and their C ABI.  The autotuner (hr_tune.cu) picks variant and
// block size per configuration.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <string>

#include "hr_host.h"
#include "hr_hop_fam.h"

using namespace hr;

namespace {

template <int REP, int PREC, int G5IN, bool CLOV = false>
__device__ __forceinline__ void hop_body(const HopArgs &a)
{
    using T = typename PrecTraits<PREC>::T;
    // nothing to do (gated off, or the solver converged); a reducing launch
    // leaves its counter clean because no block reaches the reduction
    if ((a.gate && *a.gate == 0.0) || (a.done && *a.done != 0.0)) return;
    const Geom &g = a.g;
    const int nv = g.vh << g.lrhs;
    const int stride = gridDim.x * blockDim.x;
    const T be = Real<T>::from_coef(a.beta);
    const T bu = a.g5_out ? -be : be;
    const T al = Real<T>::from_coef(a.alpha);
    SqAcc<T> red;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nv; j += stride)
        hop_site<REP, PREC, G5IN, CLOV>(a, j, al, be, bu, red);
    if (a.fin) {
        __shared__ double smem[32 * 32];
        __shared__ double sums[32];
        if (grid_reduce(red, g.nrhs, a.red, sums, smem)) finish_reduction(a.fin, sums, g.nrhs, a.scal);
    }
}

// The unrolled kernel: registers as the compiler likes (about 100 for
// double-float, two 256-thread blocks per SM) ...
template <int REP, int PREC, int G5IN>
__global__ void __launch_bounds__(256) k_hop(HopArgs a)
{
    hop_body<REP, PREC, G5IN>(a);
}

// ... and capped at 96 registers, which the double-float kernel meets without
// spilling: five 128-thread (ten 64-thread) blocks per SM instead of four,
// more warps to hide the neighbour loads.
template <int REP, int PREC, int G5IN>
__global__ void __maxnreg__(96) k_hop_r96(HopArgs a)
{
    hop_body<REP, PREC, G5IN>(a);
}

// The unrolled kernel with the clover site term in its epilogue: clover
// launches run this one (or the paired staged kernel for fundamental FP64),
// whatever the tuned shape, so that no other kernel carries the clover code.
template <int REP, int PREC, int G5IN>
__global__ void __launch_bounds__(256) k_hop_clov(HopArgs a)
{
    hop_body<REP, PREC, G5IN, true>(a);
}

// ---------------------------------------------------------------- launch

inline HopChoice default_choice(int rep, int prec)
{
    HopChoice c;
    c.variant = kVarSimple;
    c.block = (prec == kF64) ? 256 : 128;
    return c;
}

template <int REP, int PREC> struct PlainLaunch {
    static bool run(hr_ctx *ctx, const HopArgs &a, HopChoice c, int grid, cudaStream_t s, hr_status &st)
    {
        if (c.variant == kVarSimpleR96) {
            if (a.g5_in) k_hop_r96<REP, PREC, 1><<<grid, c.block, 0, s>>>(a);
            else k_hop_r96<REP, PREC, 0><<<grid, c.block, 0, s>>>(a);
            st = check_launch(ctx, "hop kernel (96 registers)");
            return true;
        }
        if (a.g5_in) k_hop<REP, PREC, 1><<<grid, c.block, 0, s>>>(a);
        else k_hop<REP, PREC, 0><<<grid, c.block, 0, s>>>(a);
        st = check_launch(ctx, "hop kernel");
        return true;
    }
};

template <int REP, int PREC> struct ClovLaunch {
    static bool run(hr_ctx *ctx, const HopArgs &a, int grid, int block, cudaStream_t s, hr_status &st)
    {
        if (a.g5_in) k_hop_clov<REP, PREC, 1><<<grid, block, 0, s>>>(a);
        else k_hop_clov<REP, PREC, 0><<<grid, block, 0, s>>>(a);
        st = check_launch(ctx, "hop kernel (clover epilogue)");
        return true;
    }
};

hr_status dispatch(hr_ctx *ctx, const Geom &g, int rep, int prec, const HopArgs &a, HopChoice c, cudaStream_t s)
{
    if (rep < 0 || rep > 2 || prec < 0 || prec > 2) return set_error(ctx, HR_ERR_INVALID_ARG, "bad rep/prec");
    const long long nv = (long long)g.vh << g.lrhs;
    if (g.twisted) {
        // twisted boundaries: one kernel for every mode, whatever the tuned shape
        hr_status st = HR_OK;
        launch_hop_twisted(ctx, rep, prec, a, s, st);
        return st;
    }
    if (a.clov_mode != kClovNone) {
        // the clover instantiations: paired staged for fundamental FP64, else unrolled
        const bool paired = rep == HR_FUND && prec == kF64;
        const int block = paired ? 256 : 128;
        const int grid = grid_for(nv, block, a.fin ? kMaxBlocks : (1 << 30));
        hr_status st = HR_OK;
        if (paired) launch_hop_clover_paired(ctx, a, grid, block, s, st);
        else for_config<ClovLaunch>(rep, prec, ctx, a, grid, block, s, st);
        return st;
    }
    // non-reducing launches cover all sites; reducing ones are capped so the
    // per-block partials fit the context's scratch
    const int grid = grid_for(nv, c.block, a.fin ? kMaxBlocks : (1 << 30));
    hr_status st = HR_OK;
    bool done = false;
    switch (c.variant) {
    case kVarStaged:
    case kVarPrefetch: done = launch_hop_staged(ctx, g, rep, prec, a, c, grid, s, st); break;
    case kVarLoop:
    case kVarLoopStaged:
    case kVarSwitch:
    case kVarSwitchStaged: done = launch_hop_looped(ctx, g, rep, prec, a, c, grid, s, st); break;
    case kVarTile:
    case kVarTileR96: done = launch_hop_tiled(ctx, g, rep, prec, a, c, grid, s, st); break;
    case kVarPaired:
    case kVarPairedStaged:
    case kVarPairedR96:
    case kVarPairedStagedR96: done = launch_hop_paired(ctx, g, rep, prec, a, c, grid, s, st); break;
    case kVarHalf:
    case kVarHalfR64:
    case kVarHalfStaged:
    case kVarHalfStagedR64:
    case kVarHalfPrefetch:
    case kVarHalfPrefetch2: done = launch_hop_half(ctx, g, rep, prec, a, c, grid, s, st); break;
    case kVarPairSites:
    case kVarPairSitesR96: done = launch_hop_pair_sites(ctx, g, rep, prec, a, c, grid, s, st); break;
    case kVarRhsChunk2:
    case kVarRhsChunk4: done = launch_hop_chunk(ctx, g, rep, prec, a, c, grid, s, st); break;
    default: break;
    }
    // the plain kernels: variants 0 and 7, and any variant without a kernel here
    if (!done) for_config<PlainLaunch>(rep, prec, ctx, a, c, grid, s, st);
    return st;
}

bool is_pow2(double x)
{
    if (!(x != 0.0)) return false;
    int e;
    double m = std::frexp(std::fabs(x), &e);
    return m == 0.5;
}

HopArgs make_args(hr_ctx *ctx, const Geom &g, const HopLaunch &L)
{
    HopArgs a;
    a.g = g;
    a.p = L.p;
    a.gauge = L.gauge;
    a.in = L.in;
    a.aux = L.aux;
    a.out = L.out;
    a.alpha = make_coef(L.alpha);
    a.beta = make_coef(L.beta);
    a.beta_pow2 = (!L.aux && is_pow2(L.beta)) ? 1 : 0;
    a.g5_in = L.g5_in;
    a.g5_out = L.g5_out;
    a.fin = L.fin;
    a.red = red_slot(ctx, C_HOP);
    a.scal = ctx->d_scal;
    a.gate = L.gate;
    a.done = L.done;
    a.unit = 1.f;
    a.nil = 0.f;
    a.cg_x = L.cg_x;
    a.cg_p = L.cg_p;
    a.cg_r = L.cg_r;
    a.inject_no_copy = ctx->inject_tile_no_copy;
    a.wait_cycles = ctx->inject_tile_no_copy ? (1LL << 20) : (1LL << 31); // ~0.5 ms / ~1 s
    a.clov = L.clov;
    a.clov_mode = L.clov ? L.clov_mode : kClovNone;
    return a;
}

} // namespace

namespace hr {

std::string tune_key(const Geom &g, int rep, int prec)
{
    char buf[128];
    snprintf(buf, sizeof buf, "hop:r%d:p%d:%dx%dx%dx%d:n%d", rep, prec, g.d[0], g.d[1], g.d[2], g.d[3], g.nrhs);
    return buf;
}

HopChoice hop_choice(hr_ctx *ctx, const Geom &g, int rep, int prec)
{
    auto it = ctx->tuned.find(tune_key(g, rep, prec));
    if (it != ctx->tuned.end()) return it->second;
    return default_choice(rep, prec);
}

std::string tune_key_fin(const Geom &g, int rep, int prec) { return tune_key(g, rep, prec) + ":fin"; }

HopChoice hop_choice_fin(hr_ctx *ctx, const Geom &g, int rep, int prec)
{
    auto it = ctx->tuned.find(tune_key_fin(g, rep, prec));
    if (it != ctx->tuned.end()) return it->second;
    return hop_choice(ctx, g, rep, prec);
}

hr_status launch_hop(hr_ctx *ctx, const Geom &g, int rep, int prec, const HopLaunch &L, cudaStream_t s)
{
    const HopChoice c = L.fin != kFinNone ? hop_choice_fin(ctx, g, rep, prec) : hop_choice(ctx, g, rep, prec);
    return dispatch(ctx, g, rep, prec, make_args(ctx, g, L), c, s);
}

hr_status launch_hop_with(hr_ctx *ctx, const Geom &g, int rep, int prec, const HopLaunch &L, HopChoice c,
                          cudaStream_t s)
{
    return dispatch(ctx, g, rep, prec, make_args(ctx, g, L), c, s);
}

bool hop_variant_available(int rep, int prec, int variant, int nrhs)
{
    // the paired kernels: fundamental (colour lanes) at every precision, adjoint
    // FP64 ((re, im) lanes; staged for quaternion links only)
    if (variant == kVarPaired) return rep == HR_FUND || prec == HR_F64;
    if (variant == kVarPairedStaged) return rep == HR_FUND || (rep == HR_ADJ && prec == HR_F64);
    // 20, 21: chunks of 2 / 4 right-hand sides per thread
    if (variant == kVarRhsChunk2) return rep == HR_FUND && prec != HR_F64 && nrhs >= 2;
    if (variant == kVarRhsChunk4) return rep == HR_FUND && prec != HR_F64 && nrhs >= 4;
    // 12 for the adjoint FP64 hop: the paired kernel with up to 168 registers
    if (variant == kVarPairedR96) return prec == HR_F64;
    if (variant == kVarPairedStagedR96) return rep == HR_FUND && prec == HR_F64;
    // the half2-projection kernels: fundamental binary16 only
    if (variant == kVarHalf || variant == kVarHalfR64 || variant == kVarHalfStaged || variant == kVarHalfStagedR64 ||
        variant == kVarHalfPrefetch || variant == kVarHalfPrefetch2)
        return rep == HR_FUND && prec == HR_F16;
    // two sites per thread: fundamental FP32 and binary16
    if (variant == kVarPairSites || variant == kVarPairSitesR96) return rep == HR_FUND && prec != HR_F64;
    // the 96-register caps spill heavily with three colours: fundamental only
    if (variant == kVarSimpleR96) return rep == HR_FUND;
    if (variant == kVarTileR96) return rep == HR_FUND && prec != HR_F16;
    if (variant == kVarTile) return prec != HR_F16;
    return variant == kVarSimple || (variant >= kVarStaged && variant < kNumHopVariants && rep != HR_ADJ_MAT);
}

// Even-site operators from two hops each:
//   Mhat    : t_o = H_oe in;        out = A in - c H_eo t_o
//   Mhat^+  : t_o = H_oe g5 in;     out = A in - c g5 H_eo t_o
//   normal  : u = Mhat in (|u|^2 reduced with fin_schur), out = Mhat^+ u
// with A = 4 + m0 and c = 1 / (4 A); with a clover field A is the site term
// (A_oo^-1 applied to t_o in the first hop's epilogue, A_ee to in in the
// second's) and c = 1/4.
hr_status apply_eo_op(hr_ctx *ctx, const Geom &g, double m0, int rep, int prec, int op, const void *gauge,
                      const void *in, void *out, void *work_odd, void *work_even, int fin_schur, const double *gate,
                      const double *done, cudaStream_t s, const CgFuse *fuse, const void *clover)
{
    // with a clover field (in the operator's clover precision):
    //   t_o = A_oo^-1 H_oe in;  out = A_ee in - 1/4 H_eo t_o
    const int cp = clover_prec(prec);
    const void *clov_inv_odd = clover_half(clover, g, rep, cp, true, 1);
    const void *clov_even = clover_half(clover, g, rep, cp, false, 0);
    const double A = 4.0 + m0, c = 1.0 / (4.0 * A);
    hr_status st;
    HopLaunch L{};
    L.gauge = gauge;
    L.gate = gate;
    L.done = done;
    auto schur = [&](const void *src, void *dst, bool dag, int fin, const CgFuse *fz) -> hr_status {
        HopLaunch h1 = L;
        h1.p = 1;
        h1.in = src;
        h1.aux = nullptr;
        h1.out = work_odd;
        h1.alpha = 0.0;
        h1.beta = 1.0;
        h1.g5_in = dag ? 1 : 0;
        h1.g5_out = 0;
        h1.fin = kFinNone;
        if (clover) {
            h1.clov = clov_inv_odd;
            h1.clov_mode = kClovOut;
        }
        hr_status e = launch_hop(ctx, g, rep, prec, h1, s);
        if (e) return e;
        HopLaunch h2 = L;
        h2.p = 0;
        h2.in = work_odd;
        h2.aux = src;
        h2.out = dst;
        h2.alpha = A;
        h2.beta = -c;
        h2.g5_in = 0;
        h2.g5_out = dag ? 1 : 0;
        h2.fin = fin;
        if (clover) {
            h2.alpha = 1.0;
            h2.beta = -0.25;
            h2.clov = clov_even;
            h2.clov_mode = kClovAux;
        }
        if (fz) {
            h2.fin = fz->fin;
            h2.cg_x = fz->x;
            h2.cg_p = fz->p;
            h2.cg_r = fz->r;
        }
        return launch_hop(ctx, g, rep, prec, h2, s);
    };
    switch (op) {
    case HR_OP_SCHUR: return schur(in, out, false, fin_schur, nullptr);
    case HR_OP_SCHUR_DAG: return schur(in, out, true, fin_schur, nullptr);
    case HR_OP_NORMAL:
        st = schur(in, work_even, false, fin_schur, nullptr);
        if (st) return st;
        return schur(work_even, out, true, kFinNone, fuse);
    }
    return set_error(ctx, HR_ERR_INVALID_ARG, "bad op %d", op);
}

} // namespace hr

extern "C" {

size_t hr_dirac_workspace_bytes(hr_lattice lat, hr_rep rep, hr_prec prec, hr_op op, int n_rhs)
{
    if (!valid_rep(rep) || !valid_prec(prec) || n_rhs < 1) return 0;
    size_t half = hr_spinor_packed_bytes(lat, rep, prec, HR_EVEN, n_rhs);
    switch (op) {
    case HR_OP_HOP: return 0;
    case HR_OP_SCHUR:
    case HR_OP_SCHUR_DAG: return half;
    case HR_OP_NORMAL: return 2 * half;
    }
    return 0;
}

hr_status hr_dirac_eo(hr_ctx *ctx, hr_lattice lat, double m0, hr_rep rep, hr_prec prec, hr_parity out_parity,
                      hr_op op, int n_rhs, const void *gauge, const void *in, void *out, void *work, size_t work_bytes,
                      hr_stream stream)
{
    if (!ctx) return HR_ERR_INVALID_ARG;
    if (!valid_rep(rep) || !valid_prec(prec)) return set_error(ctx, HR_ERR_INVALID_ARG, "bad rep/prec");
    hr_status st = validate_lattice(ctx, lat, n_rhs);
    if (st) return st;
    st = check_buffers(ctx, {gauge, in, out}, {}, {work});
    if (st) return st;
    if (in == out) return set_error(ctx, HR_ERR_INVALID_ARG, "in and out must not alias");
    if (!(4.0 + m0 != 0.0)) return set_error(ctx, HR_ERR_INVALID_ARG, "4 + m0 must be nonzero");
    Geom g = make_geom(lat, n_rhs);
    cudaStream_t s = (cudaStream_t)stream;
    if (op == HR_OP_HOP) {
        if (out_parity != HR_EVEN && out_parity != HR_ODD)
            return set_error(ctx, HR_ERR_INVALID_ARG, "HR_OP_HOP needs out_parity HR_EVEN or HR_ODD");
        HopLaunch L{};
        L.p = out_parity;
        L.gauge = gauge;
        L.in = in;
        L.out = out;
        L.beta = -0.5;
        return launch_hop(ctx, g, rep, prec, L, s);
    }
    if (op != HR_OP_SCHUR && op != HR_OP_SCHUR_DAG && op != HR_OP_NORMAL)
        return set_error(ctx, HR_ERR_INVALID_ARG, "bad op %d", (int)op);
    if (out_parity != HR_EVEN) return set_error(ctx, HR_ERR_INVALID_ARG, "Schur operators act on even sites");
    size_t need = hr_dirac_workspace_bytes(lat, rep, prec, op, n_rhs);
    if (!work || work_bytes < need)
        return set_error(ctx, HR_ERR_WORKSPACE, "workspace of %zu bytes needed, %zu given", need, work_bytes);
    size_t half = spinor_half_bytes(g, rep, prec);
    void *wo = work;
    void *we = (op == HR_OP_NORMAL) ? (char *)work + half : nullptr;
    return apply_eo_op(ctx, g, m0, rep, prec, op, gauge, in, out, wo, we, kFinNone, nullptr, nullptr, s);
}

hr_status hr_dirac_apply(hr_ctx *ctx, hr_lattice lat, double m0, hr_rep rep, hr_prec prec, const void *gauge,
                         const void *in, void *out, hr_stream stream)
{
    if (!ctx) return HR_ERR_INVALID_ARG;
    if (!valid_rep(rep) || !valid_prec(prec)) return set_error(ctx, HR_ERR_INVALID_ARG, "bad rep/prec");
    hr_status st = validate_lattice(ctx, lat, 1);
    if (st) return st;
    st = check_buffers(ctx, {gauge, in, out});
    if (st) return st;
    if (in == out) return set_error(ctx, HR_ERR_INVALID_ARG, "in and out must not alias");
    Geom g = make_geom(lat, 1);
    size_t half = spinor_half_bytes(g, rep, prec);
    cudaStream_t s = (cudaStream_t)stream;
    for (int p = 0; p < 2; ++p) {
        HopLaunch L{};
        L.p = p;
        L.gauge = gauge;
        L.in = (const char *)in + (p == 0 ? half : 0);   // the other parity
        L.aux = (const char *)in + (p == 0 ? 0 : half);  // same parity
        L.out = (char *)out + (p == 0 ? 0 : half);
        L.alpha = 4.0 + m0;
        L.beta = -0.5;
        st = launch_hop(ctx, g, rep, prec, L, s);
        if (st) return st;
    }
    return HR_OK;
}

} // extern "C"
