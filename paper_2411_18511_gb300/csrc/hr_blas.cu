// hr_blas.cu -- fused vector kernels of the CG solvers on packed spinor fields.
//
// Every kernel works site by site on the packed AoSoA layout (one thread per
// virtual site, grid-stride), so each spinor is read and written exactly once
// per call, and reductions are fused into the pass that produces the vector:
//   xr      : x += alpha p, r -= alpha q, |r|^2   (one pass, 4 reads + 2 writes)
//   p       : p = r + beta p
//   residual: r = b - Ax, |r|^2                   (reliable update / final check)
//   accum   : x_hi += x_lo, x_lo = 0              (mixed precision)
//   convert : precision change between packed layouts
// Per-RHS scalars (alpha, beta, ...) are read from the context's device scalar
// block, so a solver iteration needs no host round trip.  Reductions are FP64,
// deterministic (warp shuffle, block, then last-block sum in block order).
#include <vector>

#include "hr_host.h"

using namespace hr;

namespace {

constexpr int kBS = 256;

template <int P> using RT = typename PrecTraits<P>::T;

// arithmetic type of a kernel touching fields of two precisions: double-float
// as soon as one operand is an FP64 (double-float) field, else FP32
template <class A, class B> struct Wider { using T = A; };
template <> struct Wider<float, dd> { using T = dd; };

template <int NC, class T>
__device__ __forceinline__ void acc_site(SqAcc<T> &acc, const cpx<T> (&v)[4][NC])
{
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            acc.add(v[a][c].re);
            acc.add(v[a][c].im);
        }
}

// the right-hand side a thread works on is fixed: the grid stride is a multiple of 32
__device__ __forceinline__ int thread_rhs(const Geom &g) { return (blockIdx.x * blockDim.x + threadIdx.x) & (g.nrhs - 1); }

template <int NC, int P>
__global__ void __launch_bounds__(kBS) k_norm2(Geom g, const void *v, RedSlot red, double *scal, int fin)
{
    using T = RT<P>;
    const int nv = g.vh << g.lrhs;
    SqAcc<T> acc;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nv; j += gridDim.x * blockDim.x) {
        cpx<T> a[4][NC];
        load_spinor<NC, P>(v, g.nblk_s, j, a);
        acc_site<NC>(acc, a);
    }
    __shared__ double smem[32 * 32];
    __shared__ double sums[32];
    if (grid_reduce(acc, g.nrhs, red, sums, smem)) finish_reduction(fin, sums, g.nrhs, scal);
}

// p = r + beta p
template <int NC, int PP, int PR>
__global__ void __launch_bounds__(kBS) k_p(Geom g, void *p, const void *r, const double *scal)
{
    using T = typename Wider<RT<PP>, RT<PR>>::T;
    if (sc((double *)scal, S_FLAGS, F_DONE) != 0.0) return;
    const int nv = g.vh << g.lrhs;
    const T be = Real<T>::from_double(scal[S_BETA * kMaxRhsSlots + thread_rhs(g)]);
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nv; j += gridDim.x * blockDim.x) {
        cpx<T> pv[4][NC], rv[4][NC];
        load_spinor<NC, PP>(p, g.nblk_s, j, pv);
        load_spinor<NC, PR>(r, g.nblk_s, j, rv);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < NC; ++c) pv[a][c] = {rv[a][c].re + be * pv[a][c].re, rv[a][c].im + be * pv[a][c].im};
        store_spinor<NC, PP>(p, g.nblk_s, j, pv);
    }
}

template <int NC, int PS, int PD>
__global__ void __launch_bounds__(kBS) k_convert(Geom g, const void *src, void *dst, const double *gate)
{
    using T = typename Wider<RT<PS>, RT<PD>>::T;
    if (gate && *gate == 0.0) return;
    const int nv = g.vh << g.lrhs;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nv; j += gridDim.x * blockDim.x) {
        cpx<T> v[4][NC];
        load_spinor<NC, PS>(src, g.nblk_s, j, v);
        store_spinor<NC, PD>(dst, g.nblk_s, j, v);
    }
}

// r = b - ax (FP64 fields) ; |r|^2 -> fin ; optionally r_lo = r in precision PL
// r = b - ax in FP64 (b FP64, ax FP64 or FP32; r nullable: not stored), |r|^2 -> fin,
// and r_lo = r in the inner precision PL
template <int NC, int PL, int PA>
__global__ void __launch_bounds__(kBS) k_residual(Geom g, const void *b, const void *ax, void *r, RedSlot red,
                                                  double *scal, int fin, const double *gate, void *r_lo)
{
    using T = RT<kF64>;
    if (gate && *gate == 0.0) return;
    const int nv = g.vh << g.lrhs;
    SqAcc<T> acc;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nv; j += gridDim.x * blockDim.x) {
        cpx<T> bv[4][NC], av[4][NC];
        load_spinor<NC, kF64>(b, g.nblk_s, j, bv);
        load_spinor<NC, PA>(ax, g.nblk_s, j, av);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < NC; ++c) bv[a][c] = csub(bv[a][c], av[a][c]);
        if (r) store_spinor<NC, kF64>(r, g.nblk_s, j, bv);
        if (PL != kF64 && r_lo) store_spinor<NC, PL>(r_lo, g.nblk_s, j, bv);
        acc_site<NC>(acc, bv);
    }
    __shared__ double smem[32 * 32];
    __shared__ double sums[32];
    if (grid_reduce(acc, g.nrhs, red, sums, smem)) finish_reduction(fin, sums, g.nrhs, scal);
}

// x_hi += x_lo ; x_lo = 0  (x_hi FP64 or FP32)
template <int NC, int PH, int PL>
__global__ void __launch_bounds__(kBS) k_accum(Geom g, void *xhi, void *xlo, const double *gate)
{
    using T = RT<PH>;
    if (gate && *gate == 0.0) return;
    const int nv = g.vh << g.lrhs;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nv; j += gridDim.x * blockDim.x) {
        cpx<T> h[4][NC], l[4][NC];
        load_spinor<NC, PH>(xhi, g.nblk_s, j, h);
        load_spinor<NC, PL>(xlo, g.nblk_s, j, l);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                h[a][c] = cadd(h[a][c], l[a][c]);
                l[a][c] = {T(0.f), T(0.f)};
            }
        store_spinor<NC, PH>(xhi, g.nblk_s, j, h);
        store_spinor<NC, PL>(xlo, g.nblk_s, j, l);
    }
}

template <int NC>
__global__ void __launch_bounds__(kBS) k_axpy(Geom g, double a, const void *x, void *y)
{
    using T = RT<kF64>;
    const int nv = g.vh << g.lrhs;
    const T aa = Real<T>::from_double(a);
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nv; j += gridDim.x * blockDim.x) {
        cpx<T> xv[4][NC], yv[4][NC];
        load_spinor<NC, kF64>(x, g.nblk_s, j, xv);
        load_spinor<NC, kF64>(y, g.nblk_s, j, yv);
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int c = 0; c < NC; ++c) yv[s][c] = {yv[s][c].re + aa * xv[s][c].re, yv[s][c].im + aa * xv[s][c].im};
        store_spinor<NC, kF64>(y, g.nblk_s, j, yv);
    }
}

template <int NC>
__global__ void __launch_bounds__(kBS) k_gamma5(Geom g, void *v)
{
    using T = RT<kF64>;
    const int nv = g.vh << g.lrhs;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nv; j += gridDim.x * blockDim.x) {
        cpx<T> a[4][NC];
        load_spinor<NC, kF64>(v, g.nblk_s, j, a);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            a[0][c] = {-a[0][c].re, -a[0][c].im};
            a[1][c] = {-a[1][c].re, -a[1][c].im};
        }
        store_spinor<NC, kF64>(v, g.nblk_s, j, a);
    }
}

// per-RHS largest |component| (the hi parts of the double-float pairs) of a
// packed FP64 field, folded into scal[S_BMAX][r] as float bits: non-negative
// floats order like their bit patterns, so an unsigned atomicMax is a float max
template <int NC>
__global__ void __launch_bounds__(kBS) k_maxabs(Geom g, const void *v, double *scal)
{
    const int nv = g.vh << g.lrhs;
    float m = 0.f;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nv; j += gridDim.x * blockDim.x) {
        cpx<dd> a[4][NC];
        load_spinor<NC, kF64>(v, g.nblk_s, j, a);
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int c = 0; c < NC; ++c) m = fmaxf(m, fmaxf(fabsf(a[s][c].re.h), fabsf(a[s][c].im.h)));
    }
    // lanes of one RHS differ in their bits >= log2(nrhs)
    for (int off = 16; off >= g.nrhs; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) < g.nrhs)
        atomicMax(reinterpret_cast<unsigned *>(scal + S_BMAX * kMaxRhsSlots) + thread_rhs(g), __float_as_uint(m));
}

// scal[S_SCALE][r] = 2^-e with max = f 2^e, f in [0.5, 1); a zero field keeps 1.
// A nonzero maximum below 2^-100 raises F_RANGE: the pairs have already lost
// low bits (the low float of such a value is subnormal).
__global__ void k_scale_setup(double *scal, int nrhs)
{
    const int r = threadIdx.x;
    if (r >= nrhs) return;
    const float m = __uint_as_float(reinterpret_cast<const unsigned *>(scal + S_BMAX * kMaxRhsSlots)[r]);
    double f = 1.0;
    if (m > 0.f) {
        int e;
        frexpf(m, &e);
        f = ldexp(1.0, -e);
        if (m < 0x1p-100f) scal[S_FLAGS * kMaxRhsSlots + F_RANGE] = 1.0;
    }
    scal[S_SCALE * kMaxRhsSlots + r] = f;
}

// dst = f_r src (inverse: src / f_r), f_r a power of two: exact on both parts of a pair
template <int NC>
__global__ void __launch_bounds__(kBS) k_scale(Geom g, const void *src, void *dst, const double *scal, int inverse)
{
    const int nv = g.vh << g.lrhs;
    const int r = thread_rhs(g);
    const double f = scal[S_SCALE * kMaxRhsSlots + r];
    const float k = (float)(inverse ? 1.0 / f : f);
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nv; j += gridDim.x * blockDim.x) {
        cpx<dd> a[4][NC];
        load_spinor<NC, kF64>(src, g.nblk_s, j, a);
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                a[s][c].re = dd(a[s][c].re.h * k, a[s][c].re.l * k);
                a[s][c].im = dd(a[s][c].im.h * k, a[s][c].im.l * k);
            }
        store_spinor<NC, kF64>(dst, g.nblk_s, j, a);
    }
}

// <a, b> = sum conj(a) b over the packed FP64 fields of one parity, in FP64
// (each pair widened to a double: a utility, not a solver kernel); one
// (re, im) partial per block, summed on the host in block order
constexpr int kDotBlocks = 1024;
template <int NC>
__global__ void __launch_bounds__(kBS) k_dot(Geom g, const void *a, const void *b, double *partial)
{
    const int nv = g.vh << g.lrhs;
    double re = 0.0, im = 0.0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nv; j += gridDim.x * blockDim.x) {
        cpx<dd> u[4][NC], v[4][NC];
        load_spinor<NC, kF64>(a, g.nblk_s, j, u);
        load_spinor<NC, kF64>(b, g.nblk_s, j, v);
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const double ur = dd_to_double(u[s][c].re), ui = dd_to_double(u[s][c].im);
                const double vr = dd_to_double(v[s][c].re), vi = dd_to_double(v[s][c].im);
                re = fma(ur, vr, fma(ui, vi, re));
                im = fma(ur, vi, fma(-ui, vr, im));
            }
    }
    __shared__ double sh[2][kBS];
    sh[0][threadIdx.x] = re;
    sh[1][threadIdx.x] = im;
    __syncthreads();
    for (int w = kBS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = sh[0][0];
        partial[2 * blockIdx.x + 1] = sh[1][0];
    }
}

inline int grid_cap(hr_ctx *ctx, const Geom &g)
{
    long long nv = (long long)g.vh << g.lrhs;
    int cap = ctx->sm_count > 0 ? ctx->sm_count * 8 : 1024;
    if (cap > kMaxBlocks) cap = kMaxBlocks;
    return grid_for(nv, kBS, cap);
}

#define HR_DISPATCH_NC(rep, CALL)          \
    do {                                   \
        if (rep_nc(rep) == 2) {            \
            constexpr int NC = 2;          \
            CALL;                          \
        } else {                           \
            constexpr int NC = 3;          \
            CALL;                          \
        }                                  \
    } while (0)

#define HR_DISPATCH_P(prec, P, CALL)                       \
    do {                                                   \
        if ((prec) == kF64) { constexpr int P = kF64; CALL; } \
        else if ((prec) == kF32) { constexpr int P = kF32; CALL; } \
        else { constexpr int P = kF16; CALL; }             \
    } while (0)

} // namespace

namespace hr {

hr_status blas_norm2(hr_ctx *ctx, const Geom &g, int rep, int prec, const void *v, int fin, cudaStream_t s)
{
    int grid = grid_cap(ctx, g);
    RedSlot red = red_slot(ctx, C_NORM);
    HR_DISPATCH_NC(rep, HR_DISPATCH_P(prec, P, (k_norm2<NC, P><<<grid, kBS, 0, s>>>(g, v, red, ctx->d_scal, fin))));
    return check_launch(ctx, "norm2");
}

hr_status blas_p(hr_ctx *ctx, const Geom &g, int rep, int pp, int pr, void *p, const void *r, cudaStream_t s)
{
    int grid = grid_cap(ctx, g);
    if (pp != pr) return set_error(ctx, HR_ERR_UNSUPPORTED, "p update precision combination");
    HR_DISPATCH_NC(rep, HR_DISPATCH_P(pp, P, (k_p<NC, P, P><<<grid, kBS, 0, s>>>(g, p, r, ctx->d_scal))));
    return check_launch(ctx, "p update");
}

hr_status blas_convert(hr_ctx *ctx, const Geom &g, int rep, int psrc, int pdst, const void *src, void *dst,
                       const double *gate, cudaStream_t s)
{
    int grid = grid_cap(ctx, g);
    if (psrc == kF64) {
        HR_DISPATCH_NC(rep, HR_DISPATCH_P(pdst, P, (k_convert<NC, kF64, P><<<grid, kBS, 0, s>>>(g, src, dst, gate))));
    } else if (pdst == kF64) {
        HR_DISPATCH_NC(rep, HR_DISPATCH_P(psrc, P, (k_convert<NC, P, kF64><<<grid, kBS, 0, s>>>(g, src, dst, gate))));
    } else {
        return set_error(ctx, HR_ERR_UNSUPPORTED, "convert precision combination");
    }
    return check_launch(ctx, "convert");
}

hr_status blas_residual(hr_ctx *ctx, const Geom &g, int rep, const void *b, const void *ax, void *r, int fin,
                        const double *gate, int plo, void *r_lo, cudaStream_t s, int pax)
{
    int grid = grid_cap(ctx, g);
    RedSlot red = red_slot(ctx, C_RES);
    if (!r_lo) plo = kF64;
    if (pax == kF64) {
        HR_DISPATCH_NC(rep, HR_DISPATCH_P(plo, P, (k_residual<NC, P, kF64><<<grid, kBS, 0, s>>>(g, b, ax, r, red, ctx->d_scal, fin, gate, r_lo))));
    } else if (pax == kF32 && plo == kF16) {
        HR_DISPATCH_NC(rep, (k_residual<NC, kF16, kF32><<<grid, kBS, 0, s>>>(g, b, ax, r, red, ctx->d_scal, fin, gate, r_lo)));
    } else {
        return set_error(ctx, HR_ERR_UNSUPPORTED, "residual precision combination");
    }
    return check_launch(ctx, "residual");
}

hr_status blas_accum(hr_ctx *ctx, const Geom &g, int rep, int plo, void *xhi, void *xlo, const double *gate,
                     cudaStream_t s, int phi)
{
    int grid = grid_cap(ctx, g);
    if (plo == kF32 && phi == kF64) {
        HR_DISPATCH_NC(rep, (k_accum<NC, kF64, kF32><<<grid, kBS, 0, s>>>(g, xhi, xlo, gate)));
    } else if (plo == kF32 && phi == kF32) {
        HR_DISPATCH_NC(rep, (k_accum<NC, kF32, kF32><<<grid, kBS, 0, s>>>(g, xhi, xlo, gate)));
    } else {
        return set_error(ctx, HR_ERR_UNSUPPORTED, "accumulate precision");
    }
    return check_launch(ctx, "accumulate");
}

hr_status blas_axpy(hr_ctx *ctx, const Geom &g, int rep, double a, const void *x, void *y, cudaStream_t s)
{
    int grid = grid_cap(ctx, g);
    HR_DISPATCH_NC(rep, (k_axpy<NC><<<grid, kBS, 0, s>>>(g, a, x, y)));
    return check_launch(ctx, "axpy");
}

hr_status blas_gamma5(hr_ctx *ctx, const Geom &g, int rep, void *v, cudaStream_t s)
{
    int grid = grid_cap(ctx, g);
    HR_DISPATCH_NC(rep, (k_gamma5<NC><<<grid, kBS, 0, s>>>(g, v)));
    return check_launch(ctx, "gamma5");
}

hr_status blas_source_scale(hr_ctx *ctx, const Geom &g, int rep, const void *v, cudaStream_t s)
{
    int grid = grid_cap(ctx, g);
    HR_DISPATCH_NC(rep, (k_maxabs<NC><<<grid, kBS, 0, s>>>(g, v, ctx->d_scal)));
    hr_status st = check_launch(ctx, "max |component|");
    if (st) return st;
    k_scale_setup<<<1, 32, 0, s>>>(ctx->d_scal, g.nrhs);
    return check_launch(ctx, "source scale");
}

hr_status blas_scale(hr_ctx *ctx, const Geom &g, int rep, const void *src, void *dst, int inverse, cudaStream_t s)
{
    int grid = grid_cap(ctx, g);
    HR_DISPATCH_NC(rep, (k_scale<NC><<<grid, kBS, 0, s>>>(g, src, dst, ctx->d_scal, inverse)));
    return check_launch(ctx, "scale");
}

hr_status blas_zero(hr_ctx *ctx, const Geom &g, int rep, int prec, void *v, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(v, 0, spinor_half_bytes(g, rep, prec), s);
    if (e != cudaSuccess) return set_error(ctx, HR_ERR_CUDA, "memset: %s", cudaGetErrorString(e));
    return HR_OK;
}

hr_status blas_copy(hr_ctx *ctx, const Geom &g, int rep, int prec, const void *src, void *dst, cudaStream_t s)
{
    cudaError_t e = cudaMemcpyAsync(dst, src, spinor_half_bytes(g, rep, prec), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return set_error(ctx, HR_ERR_CUDA, "copy: %s", cudaGetErrorString(e));
    return HR_OK;
}

} // namespace hr

extern "C" {

hr_status hr_norm2(hr_ctx *ctx, hr_lattice lat, hr_rep rep, const void *v, double *result, hr_stream stream)
{
    if (!ctx) return HR_ERR_INVALID_ARG;
    if (!valid_rep(rep)) return set_error(ctx, HR_ERR_INVALID_ARG, "bad rep");
    hr_status st = validate_lattice(ctx, lat, 1);
    if (st) return st;
    if (!result) return set_error(ctx, HR_ERR_INVALID_ARG, "null pointer");
    st = check_buffers(ctx, {v});
    if (st) return st;
    Geom g = make_geom(lat, 1);
    cudaStream_t s = (cudaStream_t)stream;
    st = blas_norm2(ctx, g, rep, kF64, v, kFinStore, s);
    if (st) return st;
    cudaError_t e = cudaMemcpyAsync(ctx->h_scal, ctx->d_scal + S_OUT * kMaxRhsSlots, sizeof(double),
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_error(ctx, HR_ERR_CUDA, "norm2 readback: %s", cudaGetErrorString(e));
    *result = ctx->h_scal[0];
    return HR_OK;
}

hr_status hr_dot(hr_ctx *ctx, hr_lattice lat, hr_rep rep, const void *a, const void *b, double *re, double *im,
                 hr_stream stream)
{
    if (!ctx) return HR_ERR_INVALID_ARG;
    if (!valid_rep(rep)) return set_error(ctx, HR_ERR_INVALID_ARG, "bad rep");
    if (!re || !im) return set_error(ctx, HR_ERR_INVALID_ARG, "null result pointer");
    hr_status st = validate_lattice(ctx, lat, 1);
    if (st) return st;
    st = check_buffers(ctx, {a, b});
    if (st) return st;
    Geom g = make_geom(lat, 1);
    cudaStream_t s = (cudaStream_t)stream;
    HR_DISPATCH_NC(rep, (k_dot<NC><<<kDotBlocks, kBS, 0, s>>>(g, a, b, ctx->d_partials)));
    st = check_launch(ctx, "dot");
    if (st) return st;
    std::vector<double> h(2 * kDotBlocks);
    cudaError_t e = cudaMemcpyAsync(h.data(), ctx->d_partials, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_error(ctx, HR_ERR_CUDA, "dot readback: %s", cudaGetErrorString(e));
    double sr = 0.0, si = 0.0;
    for (int k = 0; k < kDotBlocks; ++k) {
        sr += h[2 * k];
        si += h[2 * k + 1];
    }
    *re = sr;
    *im = si;
    return HR_OK;
}

hr_status hr_axpy(hr_ctx *ctx, hr_lattice lat, hr_rep rep, double a, const void *x, void *y, hr_stream stream)
{
    if (!ctx) return HR_ERR_INVALID_ARG;
    if (!valid_rep(rep)) return set_error(ctx, HR_ERR_INVALID_ARG, "bad rep");
    hr_status st = validate_lattice(ctx, lat, 1);
    if (st) return st;
    st = check_buffers(ctx, {x, y});
    if (st) return st;
    return blas_axpy(ctx, make_geom(lat, 1), rep, a, x, y, (cudaStream_t)stream);
}

hr_status hr_gamma5(hr_ctx *ctx, hr_lattice lat, hr_rep rep, void *v, hr_stream stream)
{
    if (!ctx) return HR_ERR_INVALID_ARG;
    if (!valid_rep(rep)) return set_error(ctx, HR_ERR_INVALID_ARG, "bad rep");
    hr_status st = validate_lattice(ctx, lat, 1);
    if (st) return st;
    st = check_buffers(ctx, {v});
    if (st) return st;
    return blas_gamma5(ctx, make_geom(lat, 1), rep, v, (cudaStream_t)stream);
}

} // extern "C"
