// hr_host.h -- host-side internals of libhirep_gb300: the context, error
// reporting, argument validation and launch helpers shared by the .cu files.
#pragma once

#include <cstdarg>
#include <cstdio>
#include <cstdint>
#include <initializer_list>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "hirep_gb300.h"
#include "hr_internal.cuh"

// Device scratch owned by a context (allocated once in hr_ctx_create).
namespace hr {
constexpr int kMaxBlocks = 4096;      // cap on blocks of any reducing launch
constexpr int kMaxRhs = 32;
constexpr int kNumCounters = 64;
constexpr int kScalDoubles = 64 * kMaxRhs;

// launch shape of the hop kernel chosen by the autotuner
struct HopChoice {
    int variant; // kernel variant, 0 .. kNumHopVariants-1 (hr_hop.cu)
    int block;   // threads per block
};
constexpr int kNumHopVariants = 24;
} // namespace hr

struct hr_ctx {
    int device = 0;
    int sm_count = 0;
    std::string err;
    double *d_partials = nullptr;  // kMaxBlocks * kMaxRhs, then kRedMaxGroups * kMaxRhs group sums
    unsigned *d_counters = nullptr;
    unsigned *d_group_counters = nullptr; // kNumCounters * kRedMaxGroups (two-level reductions)
    double *d_scal = nullptr;      // kScalDoubles
    double *h_scal = nullptr;      // pinned mirror
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::map<std::string, hr::HopChoice> tuned; // autotuner: configuration key -> launch shape
    std::string tune_cache_path;                // JSON cache (HR_AUTOTUNE_CACHE), "" = none
    // instantiated CG iteration graphs, keyed by everything they bake in
    std::map<std::string, std::pair<cudaGraph_t, cudaGraphExec_t>> graphs;
    std::vector<std::string> graph_order;
    // failure injection for tests (HR_INJECT_TILE_NO_COPY=1 when the context is
    // created): the tiled hop's bulk copies are announced but never queued, so
    // its bounded waits run out (shortened to about half a millisecond)
    int inject_tile_no_copy = 0;
};
namespace hr {
constexpr size_t kMaxGraphs = 8;
}

namespace hr {

hr_status set_error(hr_ctx *ctx, hr_status st, const char *fmt, ...);
// Device buffers handed to an entry point: packed fields and work buffers are
// read and written as 16-byte vectors, canonical fields as doubles.  A null or
// misaligned one is an argument error, caught before any launch.  (nullable:
// only checked when not null.)
hr_status check_buffers(hr_ctx *ctx, std::initializer_list<const void *> packed,
                        std::initializer_list<const void *> canonical = {},
                        std::initializer_list<const void *> nullable = {});
hr_status check_launch(hr_ctx *ctx, const char *what);
hr_status validate_lattice(hr_ctx *ctx, const hr_lattice &lat, int nrhs);
bool valid_rep(int rep);
bool valid_prec(int prec);
inline int rep_nc(int rep) { return rep == HR_FUND ? 2 : 3; }

size_t spinor_half_bytes(const Geom &g, int rep, int prec);
size_t gauge_bytes(const Geom &g, int rep, int prec);

inline RedSlot red_slot(hr_ctx *ctx, int counter)
{
    RedSlot s;
    s.partials = ctx->d_partials;
    s.counter = ctx->d_counters + counter;
    s.group_counters = ctx->d_group_counters + (size_t)counter * kRedMaxGroups;
    s.group_partials = ctx->d_partials + (size_t)kMaxBlocks * kMaxRhs;
    return s;
}
static_assert(kMaxBlocks <= kRedGroup * kRedMaxGroups, "two-level reductions cover every grid");

inline int grid_for(long long n, int block, int cap)
{
    long long b = (n + block - 1) / block;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

// counters used by the reducing kernels (each reduction site has its own)
// (C_PACK: the pack status word, kPack* flags of the values packed since the
// last check, read and cleared by consume_pack_status)
enum Counter { C_HOP = 0, C_XR = 1, C_RES = 2, C_NORM = 3, C_DOT = 4, C_MISC = 5, C_BATCH = 16, C_PACK = 62,
               C_STATUS = 63 };

// clover site term in a hop epilogue (hr_clover.cuh): none, A(x) on the aux
// term (out = alpha A aux + beta acc), or A(x) on the result (out = A (alpha aux + beta acc))
enum ClovMode { kClovNone = 0, kClovAux = 1, kClovOut = 2 };

// ---- hop launches (hr_hop.cu) ----
struct HopLaunch {
    int p;                 // output parity
    const void *gauge;
    const void *in;
    const void *aux;
    void *out;
    double alpha, beta;
    int g5_in, g5_out;
    int fin;               // FinishMode of the |out|^2 reduction (kFinNone: no reduction)
    const double *gate;    // skip the launch's work unless *gate != 0 (nullable)
    const double *done;    // skip the launch's work when *done != 0 (nullable)
    // fused CG update (nullable): instead of storing out, x += alpha p and
    // r -= alpha out with alpha per RHS from the scalar block, |r|^2 -> fin
    void *cg_x;
    const void *cg_p;
    void *cg_r;
    // clover site term (nullable): the half-field of the output parity
    // (clover_half) and how the epilogue applies it (ClovMode)
    const void *clov;
    int clov_mode;
};
// a CG x/r update fused into the last hop of an operator (the operator's
// precision; x in FP32 when the operator runs in binary16)
struct CgFuse {
    void *x;
    const void *p;
    void *r;
    int fin; // kFinBeta or kFinBetaMixed
};
hr_status launch_hop(hr_ctx *ctx, const Geom &g, int rep, int prec, const HopLaunch &L, cudaStream_t s);
hr_status launch_hop_with(hr_ctx *ctx, const Geom &g, int rep, int prec, const HopLaunch &L, HopChoice c,
                          cudaStream_t s);
HopChoice hop_choice(hr_ctx *ctx, const Geom &g, int rep, int prec);
std::string tune_key(const Geom &g, int rep, int prec);
// the shape of reducing launches (aux read and |out|^2 or a fused CG update):
// their own tuned choice if there is one, else the plain one
HopChoice hop_choice_fin(hr_ctx *ctx, const Geom &g, int rep, int prec);
std::string tune_key_fin(const Geom &g, int rep, int prec);
bool hop_variant_available(int rep, int prec, int variant, int nrhs);
// autotuner cache file (hr_tune.cu)
void tune_cache_load(hr_ctx *ctx);
bool tune_cache_save(hr_ctx *ctx);
// out = op(in) on even sites, work = odd temporary (+ even temporary for NORMAL)
hr_status apply_eo_op(hr_ctx *ctx, const Geom &g, double m0, int rep, int prec, int op, const void *gauge,
                      const void *in, void *out, void *work_odd, void *work_even, int fin_schur,
                      const double *gate, const double *done, cudaStream_t s, const CgFuse *fuse = nullptr,
                      const void *clover = nullptr);

// ---- clover site term (hr_clover.cu) ----
// bytes of one of the four half-fields of a packed clover field (cp: kF64 / kF32)
size_t clover_half_bytes(const Geom &g, int rep, int cp);
// the half-field of A (inverse = false) or A^-1 on `parity`; nullptr for a null base
const void *clover_half(const void *base, const Geom &g, int rep, int cp, bool inverse, int parity);
// FP64 packed clover field -> FP32 packed clover field
hr_status clover_convert_f32(hr_ctx *ctx, const Geom &g, int rep, const void *src, void *dst, cudaStream_t s);
// out = A in on the sites of one parity, A from the half-field `half`
hr_status clover_apply_half(hr_ctx *ctx, const Geom &g, int rep, int prec, const void *half, const void *in,
                            void *out, cudaStream_t s);

// ---- BLAS launches (hr_blas.cu) ----
hr_status blas_norm2(hr_ctx *ctx, const Geom &g, int rep, int prec, const void *v, int fin, cudaStream_t s);
hr_status blas_p(hr_ctx *ctx, const Geom &g, int rep, int pp, int pr, void *p, const void *r, cudaStream_t s);
hr_status blas_convert(hr_ctx *ctx, const Geom &g, int rep, int psrc, int pdst, const void *src, void *dst,
                       const double *gate, cudaStream_t s);
// r = b - ax (FP64) with |r|^2 -> fin; also writes r in precision plo to r_lo when given
// r = b - ax (ax FP64, or FP32 with a binary16 r_lo; r nullable), |r|^2 -> fin, r_lo = r
hr_status blas_residual(hr_ctx *ctx, const Geom &g, int rep, const void *b, const void *ax, void *r, int fin,
                        const double *gate, int plo, void *r_lo, cudaStream_t s, int pax = kF64);
// packed FP64 gauge -> packed gauge of precision pdst (same rep)
hr_status gauge_convert(hr_ctx *ctx, const Geom &g, int rep, int pdst, const void *src, void *dst, cudaStream_t s);
// x_hi (FP64, or FP32) += x_lo (FP32); x_lo = 0
hr_status blas_accum(hr_ctx *ctx, const Geom &g, int rep, int plo, void *xhi, void *xlo, const double *gate,
                     cudaStream_t s, int phi = kF64);
hr_status blas_axpy(hr_ctx *ctx, const Geom &g, int rep, double a, const void *x, void *y, cudaStream_t s);
hr_status blas_gamma5(hr_ctx *ctx, const Geom &g, int rep, void *v, cudaStream_t s);
hr_status blas_zero(hr_ctx *ctx, const Geom &g, int rep, int prec, void *v, cudaStream_t s);
hr_status blas_copy(hr_ctx *ctx, const Geom &g, int rep, int prec, const void *src, void *dst, cudaStream_t s);
// per-RHS max |component| of a packed FP64 field -> scal[S_BMAX] (float bits; the slot must start at zero),
// then scal[S_SCALE] = the power of two that maps it into [0.5, 1) (1 for a zero field) and the F_RANGE
// flag when a nonzero maximum lies below 2^-100
hr_status blas_source_scale(hr_ctx *ctx, const Geom &g, int rep, const void *v, cudaStream_t s);
// dst = scal[S_SCALE] src per RHS (inverse: src / scale) on packed FP64 fields (dst may be src)
hr_status blas_scale(hr_ctx *ctx, const Geom &g, int rep, const void *src, void *dst, int inverse, cudaStream_t s);

// the pack status word (kPack* flags) since the last call, synchronising the
// stream; cleared.  HR_ERR_NUMERIC / HR_ERR_UNSUPPORTED with a message if set.
hr_status consume_pack_status(hr_ctx *ctx, cudaStream_t s);

} // namespace hr
