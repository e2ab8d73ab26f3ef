// hr_hop_loop.cu -- hop variants that run one direction body in a loop
// (generic table-driven projections, 2 and 3, or a switch over mu, 4 and 5):
// a fraction of the unrolled kernels' code, for instruction-cache-bound cases.
#include <algorithm>
#include <cstdlib>

#include "hr_hop_fam.h"

using namespace hr;

namespace {

// ---------------------------------------------------------------- looped variants
// The unrolled kernels above compile eight copies of the direction code; in
// double-float arithmetic that is tens of kilobytes of instructions and the
// warps stall on instruction fetch.  These variants run one generic direction
// body in a loop.  With k = 2 mu + (0 forward, 1 backward), the chiral-basis
// projectors of every direction take the same form
//     h_s = psi_s + i^{n_s} psi_{pi(s)}                 (s = 0, 1; pi(s) in {2, 3})
//     acc_s += r_s,  acc_{2+t} += i^{m_t} r_{sig(t)}    (r_s = U h_s, or U^+ h_s backward)
// with (pi, n, m, sig) from a table; the backward direction negates n and m
// (adds 2) and conjugates the link.  The runtime choices are integer selects
// and sign flips, which leave the FP32 pipe to the arithmetic.

// packed per-direction table (forward directions; bit fields)
//   bits 0-1 n0, 2-3 n1, 4-5 m0, 6-7 m1, 8 pi0 == 3, 9 pi1 == 3, 10 sig swaps
__device__ __constant__ unsigned c_dir_tab[4] = {
    (2u << 0) | (2u << 2) | (2u << 4) | (2u << 6) | (0u << 8) | (1u << 9) | (0u << 10), // mu = 0
    (1u << 0) | (1u << 2) | (3u << 4) | (3u << 6) | (1u << 8) | (0u << 9) | (1u << 10), // mu = 1
    (0u << 0) | (2u << 2) | (2u << 4) | (0u << 6) | (1u << 8) | (0u << 9) | (1u << 10), // mu = 2
    (1u << 0) | (3u << 2) | (3u << 4) | (1u << 6) | (0u << 8) | (1u << 9) | (0u << 10), // mu = 3
};

__device__ __forceinline__ float flip_sign(float x, bool neg)
{
    return __int_as_float(__float_as_int(x) ^ (neg ? 0x80000000 : 0));
}
__device__ __forceinline__ dd flip_sign(dd x, bool neg) { return dd(flip_sign(x.h, neg), flip_sign(x.l, neg)); }

// z * i^n for a runtime n in 0..3: a select and two sign flips
template <class T> __device__ __forceinline__ cpx<T> mul_ipow(const cpx<T> &z, int n)
{
    const bool sw = n & 1;
    T a = sw ? z.im : z.re;
    T b = sw ? z.re : z.im;
    return {flip_sign(a, n == 1 || n == 2), flip_sign(b, n >= 2)};
}

template <int REP, class T, int NC>
__device__ __forceinline__ void generic_dir(unsigned tab, bool bwd, cpx<T> (&s)[4][NC], T (&q)[4], bool neg_upper,
                                            cpx<T> (&acc)[4][NC])
{
    const int add = bwd ? 2 : 0;
    const int n0 = ((tab >> 0) + add) & 3, n1 = ((tab >> 2) + add) & 3;
    const int m0 = ((tab >> 4) + add) & 3, m1 = ((tab >> 6) + add) & 3;
    const bool p0 = (tab >> 8) & 1, p1 = (tab >> 9) & 1, sig = (tab >> 10) & 1;
    cpx<T> h[2][NC], r[2][NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        cpx<T> u0 = s[0][c], u1 = s[1][c];
        if (neg_upper) {
            u0 = {-u0.re, -u0.im};
            u1 = {-u1.re, -u1.im};
        }
        h[0][c] = cadd(u0, mul_ipow(p0 ? s[3][c] : s[2][c], n0));
        h[1][c] = cadd(u1, mul_ipow(p1 ? s[3][c] : s[2][c], n1));
    }
    // backward directions use the conjugate link: negate the vector part
    q[1] = flip_sign(q[1], bwd);
    q[2] = flip_sign(q[2], bwd);
    q[3] = flip_sign(q[3], bwd);
    if constexpr (REP == kRepFund) {
        su2_mul<false>(q, h[0], r[0]);
        su2_mul<false>(q, h[1], r[1]);
    } else {
        T R[3][3];
        quat_to_adj(q, R);
        so3_mul<false>(R, h[0], r[0]);
        so3_mul<false>(R, h[1], r[1]);
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        acc[0][c] = cadd(acc[0][c], r[0][c]);
        acc[1][c] = cadd(acc[1][c], r[1][c]);
        acc[2][c] = cadd(acc[2][c], mul_ipow(sig ? r[1][c] : r[0][c], m0));
        acc[3][c] = cadd(acc[3][c], mul_ipow(sig ? r[0][c] : r[1][c], m1));
    }
}

// even-odd index of the neighbour of direction k and of its link's site
__device__ __forceinline__ void dir_sites(const SiteNb &nb, int i, int k, int &nbr, int &link_site)
{
    const int mu = k >> 1;
    int f = nb.fwd[0], b = nb.bwd[0];
    f = (mu == 1) ? nb.fwd[1] : f;
    b = (mu == 1) ? nb.bwd[1] : b;
    f = (mu == 2) ? nb.fwd[2] : f;
    b = (mu == 2) ? nb.bwd[2] : b;
    f = (mu == 3) ? nb.fwd[3] : f;
    b = (mu == 3) ? nb.bwd[3] : b;
    const bool bwd = k & 1;
    nbr = bwd ? b : f;
    link_site = bwd ? b : i;
}

template <int REP, int PREC>
__device__ __forceinline__ void loop_issue(const HopArgs &a, const SiteNb &nb, int i, int rr, int k, uint4 *buf, int bd)
{
    using S = Stage<REP, PREC>;
    int nbr, ls;
    dir_sites(nb, i, k, nbr, ls);
    const int jn = (nbr << a.g.lrhs) + rr;
    const int lp = (k & 1) ? 1 - a.p : a.p;
    const uint4 *src = (const uint4 *)a.in;
#pragma unroll
    for (int v = 0; v < S::NV; ++v) cp_async16(buf + v * bd, src + vec_index(jn, v, S::NV));
#pragma unroll
    for (int v = 0; v < S::NQ; ++v) {
        const void *q = quat_addr<PREC>(a.gauge, a.g.nblk_g, lp, k >> 1, ls, v);
        if constexpr (PREC == kF16) cp_async8(buf + (S::NV + v) * bd, q);
        else cp_async16(buf + (S::NV + v) * bd, q);
    }
    if constexpr (PREC == kF16) {
        const float *nrm = (const float *)((const char *)a.in + SpinorLayout<S::NC, PREC>::data_bytes(a.g.nblk_s));
        cp_async4(buf + (S::NV + S::NQ) * bd, nrm + jn);
    }
}

template <int REP, int PREC, bool STAGED>
__global__ void __launch_bounds__(256) k_hop_loop(HopArgs a)
{
    using T = typename PrecTraits<PREC>::T;
    using S = Stage<REP, PREC>;
    constexpr int NC = S::NC;
    extern __shared__ uint4 stage_mem[];
    if ((a.gate && *a.gate == 0.0) || (a.done && *a.done != 0.0)) return;
    const Geom &g = a.g;
    const int nv = g.vh << g.lrhs;
    const int stride = gridDim.x * blockDim.x;
    const int bd = blockDim.x;
    uint4 *const buf0 = stage_mem + threadIdx.x;
    const int buf_step = S::NSLOT * bd; // buffer b starts at buf0 + b * buf_step
    const T be = Real<T>::from_coef(a.beta);
    const T bu = a.g5_out ? -be : be;
    const T al = Real<T>::from_coef(a.alpha);
    SqAcc<T> red;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nv; j += stride) {
        const int i = j >> g.lrhs, rr = j & (g.nrhs - 1);
        SiteNb nb;
        site_neighbours(g, i, a.p, nb);
        cpx<T> acc[4][NC];
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int c = 0; c < NC; ++c) acc[s][c] = {T(0), T(0)};
        if constexpr (STAGED) {
            loop_issue<REP, PREC>(a, nb, i, rr, 0, buf0, bd);
            cp_async_commit();
        }
#pragma unroll 1
        for (int k = 0; k < 8; ++k) {
            cpx<T> s[4][NC];
            T q[4];
            if constexpr (STAGED) {
                if (k < 7) {
                    loop_issue<REP, PREC>(a, nb, i, rr, k + 1, buf0 + ((k + 1) & 1) * buf_step, bd);
                    cp_async_commit();
                    cp_async_wait<1>();
                } else {
                    cp_async_wait<0>();
                }
                const uint4 *cur = buf0 + (k & 1) * buf_step;
                uint4 w[S::NV];
#pragma unroll
                for (int v = 0; v < S::NV; ++v) w[v] = cur[v * bd];
                float sc = 1.f;
                if constexpr (PREC == kF16) sc = *reinterpret_cast<const float *>(cur + (S::NV + S::NQ) * bd);
                spinor_from_vecs<NC, PREC>(w, sc, s);
                uint4 qv[S::NQ];
#pragma unroll
                for (int v = 0; v < S::NQ; ++v) qv[v] = cur[(S::NV + v) * bd];
                quat_from_vecs<PREC>(qv, q);
            } else {
                int nbr, ls;
                dir_sites(nb, i, k, nbr, ls);
                load_spinor<NC, PREC>(a.in, g.nblk_s, (nbr << g.lrhs) + rr, s);
                load_quat<PREC>(a.gauge, g.nblk_g, (k & 1) ? 1 - a.p : a.p, k >> 1, ls, q);
            }
            generic_dir<REP>(c_dir_tab[k >> 1], (k & 1) != 0, s, q, a.g5_in != 0, acc);
        }
        hop_epilogue<PREC>(a, j, acc, al, be, bu, red);
    }
    if (a.fin) {
        __shared__ double smem[32 * 32];
        __shared__ double sums[32];
        if (grid_reduce(red, g.nrhs, a.red, sums, smem)) finish_reduction(a.fin, sums, g.nrhs, a.scal);
    }
}

// ---------------------------------------------------------------- switched variants
// A middle way between the unrolled and the generic kernels: the loop runs over
// mu; the projection and the reconstruction of each direction are the
// compile-time code of the unrolled kernel, picked by a uniform switch, while
// the colour multiplication -- most of the arithmetic -- is compiled once for
// forward and once for backward directions.  About half the code of the
// unrolled kernel and none of the generic kernel's selects.

template <bool FWD, class T, int NC>
__device__ __forceinline__ void sw_project(int mu, const cpx<T> (&s)[4][NC], cpx<T> (&h)[2][NC])
{
    switch (mu) {
    case 0: spin_project<0, FWD>(s, h); break;
    case 1: spin_project<1, FWD>(s, h); break;
    case 2: spin_project<2, FWD>(s, h); break;
    default: spin_project<3, FWD>(s, h); break;
    }
}

template <bool FWD, class T, int NC>
__device__ __forceinline__ void sw_accumulate(int mu, cpx<T> (&acc)[4][NC], const cpx<T> (&r)[2][NC])
{
    switch (mu) {
    case 0: spin_accumulate<0, FWD>(acc, r); break;
    case 1: spin_accumulate<1, FWD>(acc, r); break;
    case 2: spin_accumulate<2, FWD>(acc, r); break;
    default: spin_accumulate<3, FWD>(acc, r); break;
    }
}

template <bool FWD, int REP, class T, int NC>
__device__ __forceinline__ void sw_direction(int mu, cpx<T> (&s)[4][NC], T (&q)[4], bool neg_upper,
                                             cpx<T> (&acc)[4][NC])
{
    if (neg_upper) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            s[0][c] = {-s[0][c].re, -s[0][c].im};
            s[1][c] = {-s[1][c].re, -s[1][c].im};
        }
    }
    cpx<T> h[2][NC], r[2][NC];
    sw_project<FWD>(mu, s, h);
    if constexpr (REP == kRepFund) {
        su2_mul<!FWD>(q, h[0], r[0]);
        su2_mul<!FWD>(q, h[1], r[1]);
    } else {
        T R[3][3];
        quat_to_adj(q, R);
        so3_mul<!FWD>(R, h[0], r[0]);
        so3_mul<!FWD>(R, h[1], r[1]);
    }
    sw_accumulate<FWD>(mu, acc, r);
}

template <int REP, int PREC, bool STAGED>
__global__ void __launch_bounds__(256) k_hop_sw(HopArgs a)
{
    using T = typename PrecTraits<PREC>::T;
    using S = Stage<REP, PREC>;
    constexpr int NC = S::NC;
    extern __shared__ uint4 stage_mem[];
    if ((a.gate && *a.gate == 0.0) || (a.done && *a.done != 0.0)) return;
    const Geom &g = a.g;
    const int nv = g.vh << g.lrhs;
    const int stride = gridDim.x * blockDim.x;
    const int bd = blockDim.x;
    uint4 *const buf0 = stage_mem + threadIdx.x;
    const int buf_step = S::NSLOT * bd;
    const T be = Real<T>::from_coef(a.beta);
    const T bu = a.g5_out ? -be : be;
    const T al = Real<T>::from_coef(a.alpha);
    SqAcc<T> red;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nv; j += stride) {
        const int i = j >> g.lrhs, rr = j & (g.nrhs - 1);
        SiteNb nb;
        site_neighbours(g, i, a.p, nb);
        cpx<T> acc[4][NC];
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int c = 0; c < NC; ++c) acc[s][c] = {T(0), T(0)};
        if constexpr (STAGED) {
            loop_issue<REP, PREC>(a, nb, i, rr, 0, buf0, bd);
            cp_async_commit();
        }
#pragma unroll 1
        for (int mu = 0; mu < 4; ++mu) {
#pragma unroll
            for (int fb = 0; fb < 2; ++fb) {
                const int k = 2 * mu + fb;
                cpx<T> s[4][NC];
                T q[4];
                if constexpr (STAGED) {
                    if (k < 7) {
                        loop_issue<REP, PREC>(a, nb, i, rr, k + 1, buf0 + ((k + 1) & 1) * buf_step, bd);
                        cp_async_commit();
                        cp_async_wait<1>();
                    } else {
                        cp_async_wait<0>();
                    }
                    const uint4 *cur = buf0 + (k & 1) * buf_step;
                    uint4 w[S::NV];
#pragma unroll
                    for (int v = 0; v < S::NV; ++v) w[v] = cur[v * bd];
                    float sc = 1.f;
                    if constexpr (PREC == kF16) sc = *reinterpret_cast<const float *>(cur + (S::NV + S::NQ) * bd);
                    spinor_from_vecs<NC, PREC>(w, sc, s);
                    uint4 qv[S::NQ];
#pragma unroll
                    for (int v = 0; v < S::NQ; ++v) qv[v] = cur[(S::NV + v) * bd];
                    quat_from_vecs<PREC>(qv, q);
                } else {
                    int nbr, ls;
                    dir_sites(nb, i, k, nbr, ls);
                    load_spinor<NC, PREC>(a.in, g.nblk_s, (nbr << g.lrhs) + rr, s);
                    load_quat<PREC>(a.gauge, g.nblk_g, fb ? 1 - a.p : a.p, mu, ls, q);
                }
                if (fb == 0) sw_direction<true, REP>(mu, s, q, a.g5_in != 0, acc);
                else sw_direction<false, REP>(mu, s, q, a.g5_in != 0, acc);
            }
        }
        hop_epilogue<PREC>(a, j, acc, al, be, bu, red);
    }
    if (a.fin) {
        __shared__ double smem[32 * 32];
        __shared__ double sums[32];
        if (grid_reduce(red, g.nrhs, a.red, sums, smem)) finish_reduction(a.fin, sums, g.nrhs, a.scal);
    }
}

template <int REP, int PREC> struct Launch {
    static bool run(hr_ctx *ctx, const Geom &, const HopArgs &a, HopChoice c, int grid, cudaStream_t s,
                    hr_status &st)
    {
        if constexpr (has_staged<REP, PREC>()) {
            const size_t sm = Stage<REP, PREC>::smem_bytes(c.block);
            const int sm_max = (int)Stage<REP, PREC>::smem_bytes(256);
            if (c.variant == kVarLoop) {
                k_hop_loop<REP, PREC, false><<<grid, c.block, 0, s>>>(a);
                st = check_launch(ctx, "looped hop kernel");
                return true;
            }
            if (c.variant == kVarLoopStaged) {
                static bool attr_set = false;
                if (!attr_set) {
                    cudaFuncSetAttribute(k_hop_loop<REP, PREC, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         sm_max);
                    attr_set = true;
                }
                k_hop_loop<REP, PREC, true><<<grid, c.block, sm, s>>>(a);
                st = check_launch(ctx, "looped staged hop kernel");
                return true;
            }
            if (c.variant == kVarSwitch) {
                k_hop_sw<REP, PREC, false><<<grid, c.block, 0, s>>>(a);
                st = check_launch(ctx, "switched hop kernel");
                return true;
            }
            if (c.variant == kVarSwitchStaged) {
                static bool attr_set2 = false;
                if (!attr_set2) {
                    cudaFuncSetAttribute(k_hop_sw<REP, PREC, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         sm_max);
                    attr_set2 = true;
                }
                k_hop_sw<REP, PREC, true><<<grid, c.block, sm, s>>>(a);
                st = check_launch(ctx, "switched staged hop kernel");
                return true;
            }
        }
        return false;
    }
};

} // namespace

namespace hr {

bool launch_hop_looped(hr_ctx *ctx, const Geom &g, int rep, int prec, const HopArgs &a, HopChoice c, int grid,
                       cudaStream_t s, hr_status &st)
{
    return for_config<Launch>(rep, prec, ctx, g, a, c, grid, s, st);
}

} // namespace hr
