// hr_core.cu -- context, error reporting, sizes and the layout-conversion
// kernels (canonical <-> packed) of libhirep_gb300.
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "hr_host.h"

using namespace hr;

// ====================================================================== errors

namespace hr {

hr_status set_error(hr_ctx *ctx, hr_status st, const char *fmt, ...)
{
    if (ctx) {
        char buf[1024];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return st;
}

hr_status check_launch(hr_ctx *ctx, const char *what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(ctx, HR_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return HR_OK;
}

bool valid_rep(int rep) { return rep == HR_FUND || rep == HR_ADJ || rep == HR_ADJ_MAT; }
bool valid_prec(int prec) { return prec == HR_F64 || prec == HR_F32 || prec == HR_F16; }

static bool lattice_ok(const hr_lattice &lat, int nrhs)
{
    long long v = 1;
    for (int k = 0; k < 4; ++k) {
        if (lat.dims[k] < 2 || (lat.dims[k] & 1)) return false;
        v *= lat.dims[k];
    }
    if (nrhs < 1 || nrhs > kMaxRhs || (nrhs & (nrhs - 1))) return false;
    if (lat.bc & ~15) return false;
    // virtual-site indices and 16-byte vector indices must fit the kernels' int arithmetic
    return (v / 2) * nrhs * 12 < (1LL << 31);
}

hr_status check_buffers(hr_ctx *ctx, std::initializer_list<const void *> packed,
                        std::initializer_list<const void *> canonical, std::initializer_list<const void *> nullable)
{
    int k = 0;
    for (const void *p : packed) {
        if (!p) return set_error(ctx, HR_ERR_INVALID_ARG, "null field pointer (argument %d)", k);
        if ((uintptr_t)p & 15u) return set_error(ctx, HR_ERR_INVALID_ARG, "packed buffer %p not 16-byte aligned", p);
        ++k;
    }
    for (const void *p : canonical) {
        if (!p) return set_error(ctx, HR_ERR_INVALID_ARG, "null field pointer");
        if ((uintptr_t)p & 7u) return set_error(ctx, HR_ERR_INVALID_ARG, "canonical buffer %p not 8-byte aligned", p);
    }
    for (const void *p : nullable)
        if (p && ((uintptr_t)p & 15u)) return set_error(ctx, HR_ERR_INVALID_ARG, "work buffer %p not 16-byte aligned", p);
    return HR_OK;
}

hr_status validate_lattice(hr_ctx *ctx, const hr_lattice &lat, int nrhs)
{
    for (int k = 0; k < 4; ++k) {
        if (lat.dims[k] < 2) return set_error(ctx, HR_ERR_INVALID_ARG, "extent %d = %d < 2", k, lat.dims[k]);
        if (lat.dims[k] & 1) return set_error(ctx, HR_ERR_UNSUPPORTED, "extent %d = %d is odd (even-odd needs even extents)", k, lat.dims[k]);
    }
    if (nrhs < 1 || nrhs > kMaxRhs || (nrhs & (nrhs - 1)))
        return set_error(ctx, HR_ERR_UNSUPPORTED, "n_rhs = %d: must be a power of two in [1, %d]", nrhs, kMaxRhs);
    if (lat.bc & ~15) return set_error(ctx, HR_ERR_INVALID_ARG, "bc = %d: one bit per direction, [0, 15]", lat.bc);
    for (int k = 0; k < 4; ++k)
        if (!std::isfinite(lat.theta[k])) return set_error(ctx, HR_ERR_INVALID_ARG, "theta[%d] is not finite", k);
    if (!lattice_ok(lat, nrhs)) return set_error(ctx, HR_ERR_UNSUPPORTED, "lattice too large for 32-bit site indexing");
    return HR_OK;
}

size_t spinor_half_bytes(const Geom &g, int rep, int prec)
{
    int nc = rep_nc(rep);
    if (nc == 2) {
        if (prec == kF64) return SpinorLayout<2, kF64>::bytes(g.nblk_s);
        if (prec == kF32) return SpinorLayout<2, kF32>::bytes(g.nblk_s);
        return SpinorLayout<2, kF16>::bytes(g.nblk_s);
    }
    if (prec == kF64) return SpinorLayout<3, kF64>::bytes(g.nblk_s);
    if (prec == kF32) return SpinorLayout<3, kF32>::bytes(g.nblk_s);
    return SpinorLayout<3, kF16>::bytes(g.nblk_s);
}

size_t gauge_bytes(const Geom &g, int rep, int prec)
{
    size_t b;
    if (rep == HR_ADJ_MAT)
        b = prec == kF64 ? GaugeMat<kF64>::bytes(g.nblk_g) : prec == kF32 ? GaugeMat<kF32>::bytes(g.nblk_g) : GaugeMat<kF16>::bytes(g.nblk_g);
    else
        b = prec == kF64 ? GaugeQuat<kF64>::bytes(g.nblk_g) : prec == kF32 ? GaugeQuat<kF32>::bytes(g.nblk_g) : GaugeQuat<kF16>::bytes(g.nblk_g);
    return (b + 255) & ~(size_t)255;
}

} // namespace hr

// ====================================================================== kernels

namespace {

// the link U_mu(x) sits on the boundary slice x_mu = L_mu - 1 of an antiperiodic direction
__device__ __forceinline__ bool boundary_link(const Geom &g, int mu, const int (&x)[4])
{
    return ((g.bc >> mu) & 1) && x[mu] == g.d[mu] - 1;
}

// one thread per link (mu, lex site).  canon (adjoint): store the representative
// of +-q with the sign bit of q0 clear, then set it on boundary links; the
// fundamental stores -q on boundary links.
template <int PREC>
__global__ void k_gauge_pack_quat(Geom g, int canon, const double *__restrict__ can, void *packed, unsigned *status)
{
    long long V = 2LL * g.vh;
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 4 * V) return;
    int mu = (int)(t / V);
    long long x = t - (long long)mu * V;
    int x3 = (int)(x % g.d[3]);
    long long r = x / g.d[3];
    int x2 = (int)(r % g.d[2]);
    r /= g.d[2];
    int x1 = (int)(r % g.d[1]);
    int x0 = (int)(r / g.d[1]);
    int p = (x0 + x1 + x2 + x3) & 1;
    int i = (int)(x >> 1);
    double a[4] = {can[t * 4 + 0], can[t * 4 + 1], can[t * 4 + 2], can[t * 4 + 3]};
    const unsigned bad = pack_range_flags(a[0]) | pack_range_flags(a[1]) | pack_range_flags(a[2]) | pack_range_flags(a[3]);
    if (bad) atomicOr(status, bad);
    const int xc[4] = {x0, x1, x2, x3};
    const bool neg = (canon && sign_bit(a[0])) != boundary_link(g, mu, xc);
    if (neg)
        for (int k = 0; k < 4; ++k) a[k] = -a[k];
    store_quat<PREC>(packed, g.nblk_g, p, mu, i, a);
}

template <int PREC>
__global__ void k_gauge_pack_mat(Geom g, const double *__restrict__ can, void *packed, unsigned *status)
{
    long long V = 2LL * g.vh;
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 4 * V) return;
    int mu = (int)(t / V);
    long long x = t - (long long)mu * V;
    int x3 = (int)(x % g.d[3]);
    long long r = x / g.d[3];
    int x2 = (int)(r % g.d[2]);
    r /= g.d[2];
    int x1 = (int)(r % g.d[1]);
    int x0 = (int)(r / g.d[1]);
    int p = (x0 + x1 + x2 + x3) & 1;
    int i = (int)(x >> 1);
    double a[4] = {can[t * 4 + 0], can[t * 4 + 1], can[t * 4 + 2], can[t * 4 + 3]};
    const unsigned bad = pack_range_flags(a[0]) | pack_range_flags(a[1]) | pack_range_flags(a[2]) | pack_range_flags(a[3]);
    if (bad) atomicOr(status, bad);
    if (sign_bit(a[0]))
        for (int k = 0; k < 4; ++k) a[k] = -a[k]; // R(q) = R(-q); quat_to_adj reads the sign bit
    double R[3][3];
    quat_to_adj(a, R);
    const int xc[4] = {x0, x1, x2, x3};
    const double sg = boundary_link(g, mu, xc) ? -1.0 : 1.0;
    for (int e = 0; e < 9; ++e) {
        store_mat_entry<PREC>(packed, g.nblk_g, p, mu, i, e, sg * R[e / 3][e % 3]);
    }
}

// canonical double[nrhs][V][4][NC][2] -> packed virtual sites of parity p.
// One thread per (rhs, even-odd site).
template <int NC, int PREC>
__global__ void k_spinor_pack(Geom g, int p, const double *__restrict__ can, void *packed, unsigned *status)
{
    using T = double; // the canonical side is FP64; the layout code converts
    long long n = (long long)g.vh << g.lrhs;
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    int r = (int)(t / g.vh);
    int i = (int)(t - (long long)r * g.vh);
    long long lex = eo_to_lex(g, i, p);
    long long V = 2LL * g.vh;
    const double *src = can + ((long long)r * V + lex) * (8 * NC);
    cpx<T> s[4][NC];
    unsigned bad = 0;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            s[a][c] = {(T)src[(a * NC + c) * 2], (T)src[(a * NC + c) * 2 + 1]};
            bad |= pack_range_flags(s[a][c].re) | pack_range_flags(s[a][c].im);
        }
    if (bad) atomicOr(status, bad);
    store_spinor<NC, PREC>(packed, g.nblk_s, (i << g.lrhs) + r, s);
}

template <int NC, int PREC>
__global__ void k_spinor_unpack(Geom g, int p, const void *packed, double *__restrict__ can)
{
    using T = double; // the canonical side is FP64; the layout code converts
    long long n = (long long)g.vh << g.lrhs;
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    int r = (int)(t / g.vh);
    int i = (int)(t - (long long)r * g.vh);
    long long lex = eo_to_lex(g, i, p);
    long long V = 2LL * g.vh;
    double *dst = can + ((long long)r * V + lex) * (8 * NC);
    cpx<T> s[4][NC];
    load_spinor<NC, PREC>(packed, g.nblk_s, (i << g.lrhs) + r, s);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            dst[(a * NC + c) * 2] = (double)s[a][c].re;
            dst[(a * NC + c) * 2 + 1] = (double)s[a][c].im;
        }
}

template <int NC, int PREC>
hr_status launch_spinor_pack(hr_ctx *ctx, const Geom &g, int p, const double *can, void *packed, bool unpack,
                             cudaStream_t s)
{
    long long n = (long long)g.vh << g.lrhs;
    int bs = 256;
    int grid = (int)((n + bs - 1) / bs);
    if (unpack) k_spinor_unpack<NC, PREC><<<grid, bs, 0, s>>>(g, p, packed, (double *)can);
    else k_spinor_pack<NC, PREC><<<grid, bs, 0, s>>>(g, p, can, packed, ctx->d_counters + C_PACK);
    return check_launch(ctx, unpack ? "spinor unpack" : "spinor pack");
}

hr_status spinor_convert(hr_ctx *ctx, hr_lattice lat, int rep, int prec, int parity, int n_rhs, const double *can,
                         void *packed, bool unpack, cudaStream_t s)
{
    if (!ctx) return HR_ERR_INVALID_ARG;
    if (!valid_rep(rep) || !valid_prec(prec)) return set_error(ctx, HR_ERR_INVALID_ARG, "bad rep/prec");
    if (parity < 0 || parity > 2) return set_error(ctx, HR_ERR_INVALID_ARG, "bad parity %d", parity);
    hr_status st = validate_lattice(ctx, lat, n_rhs);
    if (st) return st;
    st = check_buffers(ctx, {packed}, {can});
    if (st) return st;
    Geom g = make_geom(lat, n_rhs);
    size_t half = spinor_half_bytes(g, rep, prec);
    int nc = rep_nc(rep);
    for (int p = 0; p < 2; ++p) {
        if (parity != HR_FULL && parity != p) continue;
        char *dst = (char *)packed + ((parity == HR_FULL && p == 1) ? half : 0);
        if (nc == 2) {
            if (prec == kF64) st = launch_spinor_pack<2, kF64>(ctx, g, p, can, dst, unpack, s);
            else if (prec == kF32) st = launch_spinor_pack<2, kF32>(ctx, g, p, can, dst, unpack, s);
            else st = launch_spinor_pack<2, kF16>(ctx, g, p, can, dst, unpack, s);
        } else {
            if (prec == kF64) st = launch_spinor_pack<3, kF64>(ctx, g, p, can, dst, unpack, s);
            else if (prec == kF32) st = launch_spinor_pack<3, kF32>(ctx, g, p, can, dst, unpack, s);
            else st = launch_spinor_pack<3, kF16>(ctx, g, p, can, dst, unpack, s);
        }
        if (st) return st;
    }
    return HR_OK;
}

// packed FP64 gauge -> packed gauge of precision PD, one thread per (p, mu, site)
template <int PD, bool MAT>
__global__ void k_gauge_convert(Geom g, const void *src, void *dst)
{
    long long n = 8LL * g.nblk_g * 32;
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    size_t slot = (size_t)(t >> 5);
    int lane = (int)(t & 31);
    if (MAT) {
        for (int e = 0; e < 9; ++e) {
            size_t idx = (slot * 9 + e) * 32 + lane;
            float2 w = ((const float2 *)src)[idx];
            float v = __fadd_rn(w.x, w.y);
            if (PD == kF32) ((float *)dst)[idx] = v;
            else ((__half *)dst)[idx] = __float2half_rn(v);
        }
    } else {
        // FP64 packed links are double-float pairs: hi float4 then lo float4
        const float4 *q = (const float4 *)src;
        float4 hi = q[(slot * 2 + 0) * 32 + lane], lo = q[(slot * 2 + 1) * 32 + lane];
        // the sign of hi survives (-0 + 0 would round to +0 and lose the
        // adjoint links' boundary bit on a link with q0 = 0)
        float4 w0 = make_float4(copysignf(__fadd_rn(hi.x, lo.x), hi.x), copysignf(__fadd_rn(hi.y, lo.y), hi.y),
                                copysignf(__fadd_rn(hi.z, lo.z), hi.z), copysignf(__fadd_rn(hi.w, lo.w), hi.w));
        if (PD == kF32) {
            ((float4 *)dst)[slot * 32 + lane] = w0;
        } else {
            __half2 h0 = __floats2half2_rn(w0.x, w0.y);
            __half2 h1 = __floats2half2_rn(w0.z, w0.w);
            uint2 w;
            w.x = *reinterpret_cast<uint32_t *>(&h0);
            w.y = *reinterpret_cast<uint32_t *>(&h1);
            ((uint2 *)dst)[slot * 32 + lane] = w;
        }
    }
}

} // namespace

namespace hr {
hr_status consume_pack_status(hr_ctx *ctx, cudaStream_t s)
{
    unsigned flags = 0;
    cudaError_t e = cudaMemcpyAsync(&flags, ctx->d_counters + C_PACK, sizeof flags, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && flags) e = cudaMemsetAsync(ctx->d_counters + C_PACK, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(ctx, HR_ERR_CUDA, "pack status readback: %s", cudaGetErrorString(e));
    }
    if (flags & kPackNonFinite) return set_error(ctx, HR_ERR_NUMERIC, "a packed field held a NaN or Inf");
    if (flags & kPackAboveRange)
        return set_error(ctx, HR_ERR_UNSUPPORTED,
                         "a packed value exceeded 2^120 = 1.3e36 in magnitude (the pair-of-floats FP64 layout "
                         "keeps the float exponent range): scale the field down");
    return HR_OK;
}

hr_status gauge_convert(hr_ctx *ctx, const Geom &g, int rep, int pdst, const void *src, void *dst, cudaStream_t s)
{
    long long n = 8LL * g.nblk_g * 32;
    int bs = 256;
    int grid = (int)((n + bs - 1) / bs);
    bool mat = rep == HR_ADJ_MAT;
    if (pdst == kF32) {
        if (mat) k_gauge_convert<kF32, true><<<grid, bs, 0, s>>>(g, src, dst);
        else k_gauge_convert<kF32, false><<<grid, bs, 0, s>>>(g, src, dst);
    } else if (pdst == kF16) {
        if (mat) k_gauge_convert<kF16, true><<<grid, bs, 0, s>>>(g, src, dst);
        else k_gauge_convert<kF16, false><<<grid, bs, 0, s>>>(g, src, dst);
    } else {
        return set_error(ctx, HR_ERR_UNSUPPORTED, "gauge convert target precision");
    }
    return check_launch(ctx, "gauge convert");
}
} // namespace hr

// ====================================================================== C ABI

extern "C" {

const char *hr_version(void) { return "hirep_gb300 0.1 (sm_103a)"; }

double hr_kappa_to_m0(double kappa) { return 1.0 / (2.0 * kappa) - 4.0; }
double hr_m0_to_kappa(double m0) { return 1.0 / (8.0 + 2.0 * m0); }

hr_status hr_ctx_create(hr_ctx **out, int device)
{
    if (!out) return HR_ERR_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return HR_ERR_CUDA;
    }
    hr_ctx *ctx = new hr_ctx();
    ctx->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_partials, sizeof(double) * (kMaxBlocks + kRedMaxGroups) * kMaxRhs);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_counters, sizeof(unsigned) * kNumCounters);
    if (e == cudaSuccess) e = cudaMemset(ctx->d_counters, 0, sizeof(unsigned) * kNumCounters);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_group_counters, sizeof(unsigned) * kNumCounters * kRedMaxGroups);
    if (e == cudaSuccess) e = cudaMemset(ctx->d_group_counters, 0, sizeof(unsigned) * kNumCounters * kRedMaxGroups);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_scal, sizeof(double) * kScalDoubles);
    if (e == cudaSuccess) e = cudaMemset(ctx->d_scal, 0, sizeof(double) * kScalDoubles);
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_scal, sizeof(double) * kScalDoubles);
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev1);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaGetLastError();
        hr_ctx_destroy(ctx);
        return HR_ERR_CUDA;
    }
    const char *path = getenv("HR_AUTOTUNE_CACHE");
    if (path && path[0]) {
        ctx->tune_cache_path = path;
        tune_cache_load(ctx);
    }
    const char *inj = getenv("HR_INJECT_TILE_NO_COPY");
    ctx->inject_tile_no_copy = (inj && inj[0] == '1') ? 1 : 0;
    *out = ctx;
    return HR_OK;
}

hr_status hr_ctx_destroy(hr_ctx *ctx)
{
    if (!ctx) return HR_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    if (ctx->d_partials) cudaFree(ctx->d_partials);
    if (ctx->d_counters) cudaFree(ctx->d_counters);
    if (ctx->d_group_counters) cudaFree(ctx->d_group_counters);
    if (ctx->d_scal) cudaFree(ctx->d_scal);
    if (ctx->h_scal) cudaFreeHost(ctx->h_scal);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    for (auto &kv : ctx->graphs) {
        cudaGraphExecDestroy(kv.second.second);
        cudaGraphDestroy(kv.second.first);
    }
    delete ctx;
    return HR_OK;
}

hr_status hr_ctx_status(hr_ctx *ctx, hr_stream stream)
{
    if (!ctx) return HR_ERR_INVALID_ARG;
    return consume_pack_status(ctx, (cudaStream_t)stream);
}

const char *hr_last_error(const hr_ctx *ctx)
{
    if (!ctx) return "null context";
    return ctx->err.c_str();
}

size_t hr_gauge_packed_bytes(hr_lattice lat, hr_rep rep, hr_prec prec)
{
    if (!valid_rep(rep) || !valid_prec(prec) || !lattice_ok(lat, 1)) return 0;
    return gauge_bytes(make_geom(lat, 1), rep, prec);
}

size_t hr_spinor_packed_bytes(hr_lattice lat, hr_rep rep, hr_prec prec, hr_parity parity, int n_rhs)
{
    if (!valid_rep(rep) || !valid_prec(prec) || !lattice_ok(lat, n_rhs)) return 0;
    if (parity < 0 || parity > 2) return 0;
    size_t half = spinor_half_bytes(make_geom(lat, n_rhs), rep, prec);
    return parity == HR_FULL ? 2 * half : half;
}

hr_status hr_gauge_pack(hr_ctx *ctx, hr_lattice lat, hr_rep rep, hr_prec prec, const double *canonical, void *packed,
                        hr_stream stream)
{
    if (!ctx) return HR_ERR_INVALID_ARG;
    if (!valid_rep(rep) || !valid_prec(prec)) return set_error(ctx, HR_ERR_INVALID_ARG, "bad rep/prec");
    hr_status st = validate_lattice(ctx, lat, 1);
    if (st) return st;
    st = check_buffers(ctx, {packed}, {canonical});
    if (st) return st;
    Geom g = make_geom(lat, 1);
    cudaStream_t s = (cudaStream_t)stream;
    // zero the padding lanes so packed buffers are fully defined
    cudaMemsetAsync(packed, 0, gauge_bytes(g, rep, prec), s);
    long long n = 8LL * g.vh;
    int bs = 256;
    int grid = (int)((n + bs - 1) / bs);
    unsigned *status = ctx->d_counters + C_PACK;
    if (rep == HR_ADJ_MAT) {
        if (prec == kF64) k_gauge_pack_mat<kF64><<<grid, bs, 0, s>>>(g, canonical, packed, status);
        else if (prec == kF32) k_gauge_pack_mat<kF32><<<grid, bs, 0, s>>>(g, canonical, packed, status);
        else k_gauge_pack_mat<kF16><<<grid, bs, 0, s>>>(g, canonical, packed, status);
    } else {
        const int canon = rep == HR_ADJ ? 1 : 0;
        if (prec == kF64) k_gauge_pack_quat<kF64><<<grid, bs, 0, s>>>(g, canon, canonical, packed, status);
        else if (prec == kF32) k_gauge_pack_quat<kF32><<<grid, bs, 0, s>>>(g, canon, canonical, packed, status);
        else k_gauge_pack_quat<kF16><<<grid, bs, 0, s>>>(g, canon, canonical, packed, status);
    }
    return check_launch(ctx, "gauge pack");
}

hr_status hr_spinor_pack(hr_ctx *ctx, hr_lattice lat, hr_rep rep, hr_prec prec, hr_parity parity, int n_rhs,
                         const double *canonical, void *packed, hr_stream stream)
{
    if (ctx && packed && valid_rep(rep) && valid_prec(prec) && lattice_ok(lat, n_rhs) && parity >= 0 && parity <= 2)
        cudaMemsetAsync(packed, 0, hr_spinor_packed_bytes(lat, rep, prec, parity, n_rhs), (cudaStream_t)stream);
    return spinor_convert(ctx, lat, rep, prec, parity, n_rhs, canonical, packed, false, (cudaStream_t)stream);
}

hr_status hr_spinor_unpack(hr_ctx *ctx, hr_lattice lat, hr_rep rep, hr_prec prec, hr_parity parity, int n_rhs,
                           const void *packed, double *canonical, hr_stream stream)
{
    return spinor_convert(ctx, lat, rep, prec, parity, n_rhs, canonical, (void *)packed, true,
                          (cudaStream_t)stream);
}

} // extern "C"
