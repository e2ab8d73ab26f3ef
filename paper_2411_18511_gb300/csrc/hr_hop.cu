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
// Two variants of the same arithmetic:
//   k_hop        loads each direction's operands straight into registers;
//   k_hop_staged copies direction k+1's spinor and link into shared memory with
//                cp.async while direction k is computed (double buffer, one
//                thread's own slots, no block barrier), so memory latency
//                overlaps the arithmetic without costing registers.
// The autotuner (hr_autotune) picks variant and block size per configuration.
#include <cstdlib>
#include <cstring>
#include <string>

#include "hr_host.h"
#include "hr_hop_dev.cuh"

using namespace hr;

namespace {

template <int REP, int PREC>
__global__ void __launch_bounds__(256) k_hop(HopArgs a)
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
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nv; j += stride) hop_site<REP, PREC>(a, j, al, be, bu, red);
    if (a.fin) {
        __shared__ double smem[32 * 32];
        __shared__ double sums[32];
        if (grid_reduce(red.get(), g.nrhs, a.red, sums, smem)) finish_reduction(a.fin, sums, g.nrhs, a.scal);
    }
}

// ---------------------------------------------------------------- staged variant

template <int REP, int PREC> struct Stage {
    static constexpr int NC = RepTraits<REP>::NC;
    static constexpr int NV = SpinorLayout<NC, PREC>::NVEC;
    static constexpr int NQ = QuatSlots<PREC>::n;
    static constexpr int NSLOT = NV + NQ + (PREC == kF16 ? 1 : 0); // 16-byte slots per direction
    static size_t smem_bytes(int block) { return (size_t)2 * NSLOT * block * 16; }
};

// direction K = 2 mu + (0 forward, 1 backward): queue its operands' copies
template <int K, int REP, int PREC>
__device__ __forceinline__ void stage_issue(const HopArgs &a, int i, int rr, const SiteNb &nb, uint4 *buf, int bd)
{
    using S = Stage<REP, PREC>;
    constexpr int MU = K >> 1;
    constexpr bool FWD = (K & 1) == 0;
    const int jn = ((FWD ? nb.fwd[MU] : nb.bwd[MU]) << a.g.lrhs) + rr;
    const int site_link = FWD ? i : nb.bwd[MU];
    const int link_par = FWD ? a.p : 1 - a.p;
    const uint4 *src = (const uint4 *)a.in;
#pragma unroll
    for (int v = 0; v < S::NV; ++v) cp_async16(buf + v * bd, src + vec_index(jn, v, S::NV));
#pragma unroll
    for (int v = 0; v < S::NQ; ++v) {
        const void *q = quat_addr<PREC>(a.gauge, a.g.nblk_g, link_par, MU, site_link, v);
        if constexpr (PREC == kF16) cp_async8(buf + (S::NV + v) * bd, q);
        else cp_async16(buf + (S::NV + v) * bd, q);
    }
    if constexpr (PREC == kF16) {
        const float *nrm = (const float *)((const char *)a.in + SpinorLayout<S::NC, PREC>::data_bytes(a.g.nblk_s));
        cp_async4(buf + (S::NV + S::NQ) * bd, nrm + jn);
    }
}

template <int K, int REP, int PREC, class T, int NC>
__device__ __forceinline__ void stage_compute(const HopArgs &a, const uint4 *buf, int bd, cpx<T> (&acc)[4][NC])
{
    using S = Stage<REP, PREC>;
    constexpr int MU = K >> 1;
    constexpr bool FWD = (K & 1) == 0;
    uint4 w[S::NV];
#pragma unroll
    for (int v = 0; v < S::NV; ++v) w[v] = buf[v * bd];
    float sc = 1.f;
    if constexpr (PREC == kF16) sc = *reinterpret_cast<const float *>(buf + (S::NV + S::NQ) * bd);
    cpx<T> s[4][NC];
    spinor_from_vecs<NC, PREC>(w, sc, s);
    uint4 qv[S::NQ];
#pragma unroll
    for (int v = 0; v < S::NQ; ++v) qv[v] = buf[(S::NV + v) * bd];
    T q[4];
    quat_from_vecs<PREC>(qv, q);
    if constexpr (REP == kRepFund) {
        hop_compute<MU, FWD, REP>(s, q, a.g5_in != 0, acc);
    } else {
        T R[3][3];
        quat_to_adj(q, R);
        hop_compute<MU, FWD, REP>(s, R, a.g5_in != 0, acc);
    }
}

// one pipeline step: queue direction K+1 into the other buffer, wait for K, compute K
template <int K, int REP, int PREC, class T, int NC>
__device__ __forceinline__ void stage_step(const HopArgs &a, int i, int rr, const SiteNb &nb, uint4 *b0, uint4 *b1,
                                           int bd, cpx<T> (&acc)[4][NC])
{
    uint4 *cur = (K & 1) ? b1 : b0;
    uint4 *nxt = (K & 1) ? b0 : b1;
    if constexpr (K < 7) {
        stage_issue<K + 1, REP, PREC>(a, i, rr, nb, nxt, bd);
        cp_async_commit();
        cp_async_wait<1>();
    } else {
        cp_async_wait<0>();
    }
    stage_compute<K, REP, PREC>(a, cur, bd, acc);
}

template <int REP, int PREC>
__global__ void __launch_bounds__(256) k_hop_staged(HopArgs a)
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
    // this thread's slots: [buffer][slot][thread], consecutive threads -> consecutive 16 B
    uint4 *b0 = stage_mem + threadIdx.x;
    uint4 *b1 = stage_mem + S::NSLOT * bd + threadIdx.x;
    const T be = Real<T>::from_coef(a.beta);
    const T bu = a.g5_out ? -be : be;
    const T al = Real<T>::from_coef(a.alpha);
    SqAcc<T> red;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nv; j += stride) {
        const int i = j >> g.lrhs, rr = j & (g.nrhs - 1);
        SiteNb nb;
        site_neighbours(g, i, a.p, nb);
        stage_issue<0, REP, PREC>(a, i, rr, nb, b0, bd);
        cp_async_commit();
        cpx<T> acc[4][NC];
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int c = 0; c < NC; ++c) acc[s][c] = {T(0), T(0)};
        stage_step<0, REP, PREC>(a, i, rr, nb, b0, b1, bd, acc);
        stage_step<1, REP, PREC>(a, i, rr, nb, b0, b1, bd, acc);
        stage_step<2, REP, PREC>(a, i, rr, nb, b0, b1, bd, acc);
        stage_step<3, REP, PREC>(a, i, rr, nb, b0, b1, bd, acc);
        stage_step<4, REP, PREC>(a, i, rr, nb, b0, b1, bd, acc);
        stage_step<5, REP, PREC>(a, i, rr, nb, b0, b1, bd, acc);
        stage_step<6, REP, PREC>(a, i, rr, nb, b0, b1, bd, acc);
        stage_step<7, REP, PREC>(a, i, rr, nb, b0, b1, bd, acc);
        hop_epilogue<PREC>(a, j, acc, al, be, bu, red);
    }
    if (a.fin) {
        __shared__ double smem[32 * 32];
        __shared__ double sums[32];
        if (grid_reduce(red.get(), g.nrhs, a.red, sums, smem)) finish_reduction(a.fin, sums, g.nrhs, a.scal);
    }
}

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
        if (grid_reduce(red.get(), g.nrhs, a.red, sums, smem)) finish_reduction(a.fin, sums, g.nrhs, a.scal);
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
        if (grid_reduce(red.get(), g.nrhs, a.red, sums, smem)) finish_reduction(a.fin, sums, g.nrhs, a.scal);
    }
}

// ---------------------------------------------------------------- prefetching variant
// Unrolled like k_hop, but the operands of direction k+1 are loaded into a
// second set of registers before direction k is computed, so every load has a
// whole direction of arithmetic to arrive in.  Costs registers (two operand
// sets) and so occupancy; the autotuner decides whether it pays.

template <int K, int REP, int PREC, class T, int NC>
__device__ __forceinline__ void pf_load(const HopArgs &a, int i, int rr, const SiteNb &nb, cpx<T> (&s)[4][NC],
                                        T (&q)[4], float &sc)
{
    constexpr int MU = K >> 1;
    constexpr bool FWD = (K & 1) == 0;
    const int nbr = FWD ? nb.fwd[MU] : nb.bwd[MU];
    load_spinor_raw<NC, PREC>(a.in, a.g.nblk_s, (nbr << a.g.lrhs) + rr, s, sc);
    load_quat<PREC>(a.gauge, a.g.nblk_g, FWD ? a.p : 1 - a.p, MU, FWD ? i : nb.bwd[MU], q);
}

template <int K, int REP, int PREC, class T, int NC>
__device__ __forceinline__ void pf_compute(const HopArgs &a, cpx<T> (&s)[4][NC], T (&q)[4], float sc,
                                           cpx<T> (&acc)[4][NC])
{
    constexpr int MU = K >> 1;
    constexpr bool FWD = (K & 1) == 0;
    if constexpr (REP == kRepFund) {
        if constexpr (PREC == kF16) {
#pragma unroll
            for (int k = 0; k < 4; ++k) q[k] = q[k] * sc;
        }
        hop_compute<MU, FWD, REP>(s, q, a.g5_in != 0, acc);
    } else {
        T R[3][3];
        quat_to_adj(q, R);
        if constexpr (PREC == kF16) {
#pragma unroll
            for (int k = 0; k < 9; ++k) R[k / 3][k % 3] = R[k / 3][k % 3] * sc;
        }
        hop_compute<MU, FWD, REP>(s, R, a.g5_in != 0, acc);
    }
}

template <int REP, int PREC>
__global__ void __launch_bounds__(256) k_hop_pf(HopArgs a)
{
    using T = typename PrecTraits<PREC>::T;
    constexpr int NC = RepTraits<REP>::NC;
    if ((a.gate && *a.gate == 0.0) || (a.done && *a.done != 0.0)) return;
    const Geom &g = a.g;
    const int nv = g.vh << g.lrhs;
    const int stride = gridDim.x * blockDim.x;
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
        cpx<T> sA[4][NC], sB[4][NC];
        T qA[4], qB[4];
        float cA, cB;
        pf_load<0, REP, PREC>(a, i, rr, nb, sA, qA, cA);
        pf_load<1, REP, PREC>(a, i, rr, nb, sB, qB, cB);
        pf_compute<0, REP, PREC>(a, sA, qA, cA, acc);
        pf_load<2, REP, PREC>(a, i, rr, nb, sA, qA, cA);
        pf_compute<1, REP, PREC>(a, sB, qB, cB, acc);
        pf_load<3, REP, PREC>(a, i, rr, nb, sB, qB, cB);
        pf_compute<2, REP, PREC>(a, sA, qA, cA, acc);
        pf_load<4, REP, PREC>(a, i, rr, nb, sA, qA, cA);
        pf_compute<3, REP, PREC>(a, sB, qB, cB, acc);
        pf_load<5, REP, PREC>(a, i, rr, nb, sB, qB, cB);
        pf_compute<4, REP, PREC>(a, sA, qA, cA, acc);
        pf_load<6, REP, PREC>(a, i, rr, nb, sA, qA, cA);
        pf_compute<5, REP, PREC>(a, sB, qB, cB, acc);
        pf_load<7, REP, PREC>(a, i, rr, nb, sB, qB, cB);
        pf_compute<6, REP, PREC>(a, sA, qA, cA, acc);
        pf_compute<7, REP, PREC>(a, sB, qB, cB, acc);
        hop_epilogue<PREC>(a, j, acc, al, be, bu, red);
    }
    if (a.fin) {
        __shared__ double smem[32 * 32];
        __shared__ double sums[32];
        if (grid_reduce(red.get(), g.nrhs, a.red, sums, smem)) finish_reduction(a.fin, sums, g.nrhs, a.scal);
    }
}

// ---------------------------------------------------------------- launch

constexpr int kVarSimple = 0, kVarStaged = 1, kVarLoop = 2, kVarLoopStaged = 3, kVarSwitch = 4,
              kVarSwitchStaged = 5, kVarPrefetch = 6;
constexpr int kNumVariants = 7;

template <int REP, int PREC> constexpr bool has_staged() { return REP != kRepAdjMat; }

// default choice before (or without) autotuning: the unrolled kernel (256
// threads for double-float, 128 otherwise), the fastest on GB300 without tuning
inline HopChoice default_choice(int rep, int prec)
{
    HopChoice c;
    c.variant = kVarSimple;
    c.block = (prec == kF64) ? 256 : 128;
    return c;
}

template <int REP, int PREC>
hr_status launch_t(hr_ctx *ctx, const Geom &g, const HopArgs &a, HopChoice c, cudaStream_t s)
{
    const long long nv = (long long)g.vh << g.lrhs;
    // non-reducing launches cover all sites; reducing ones are capped so the
    // per-block partials fit the context's scratch
    int cap = a.fin ? kMaxBlocks : (1 << 30);
    int grid = grid_for(nv, c.block, cap);
    if constexpr (has_staged<REP, PREC>()) {
        const size_t sm = Stage<REP, PREC>::smem_bytes(c.block);
        const int sm_max = (int)Stage<REP, PREC>::smem_bytes(256);
        if (c.variant == kVarStaged) {
            static bool attr_set = false;
            if (!attr_set) {
                cudaFuncSetAttribute(k_hop_staged<REP, PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_max);
                attr_set = true;
            }
            k_hop_staged<REP, PREC><<<grid, c.block, sm, s>>>(a);
            return check_launch(ctx, "staged hop kernel");
        }
        if (c.variant == kVarLoop) {
            k_hop_loop<REP, PREC, false><<<grid, c.block, 0, s>>>(a);
            return check_launch(ctx, "looped hop kernel");
        }
        if (c.variant == kVarLoopStaged) {
            static bool attr_set2 = false;
            if (!attr_set2) {
                cudaFuncSetAttribute(k_hop_loop<REP, PREC, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_max);
                attr_set2 = true;
            }
            k_hop_loop<REP, PREC, true><<<grid, c.block, sm, s>>>(a);
            return check_launch(ctx, "looped staged hop kernel");
        }
        if (c.variant == kVarSwitch) {
            k_hop_sw<REP, PREC, false><<<grid, c.block, 0, s>>>(a);
            return check_launch(ctx, "switched hop kernel");
        }
        if (c.variant == kVarPrefetch) {
            k_hop_pf<REP, PREC><<<grid, c.block, 0, s>>>(a);
            return check_launch(ctx, "prefetching hop kernel");
        }
        if (c.variant == kVarSwitchStaged) {
            static bool attr_set3 = false;
            if (!attr_set3) {
                cudaFuncSetAttribute(k_hop_sw<REP, PREC, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_max);
                attr_set3 = true;
            }
            k_hop_sw<REP, PREC, true><<<grid, c.block, sm, s>>>(a);
            return check_launch(ctx, "switched staged hop kernel");
        }
    }
    k_hop<REP, PREC><<<grid, c.block, 0, s>>>(a);
    return check_launch(ctx, "hop kernel");
}

hr_status dispatch(hr_ctx *ctx, const Geom &g, int rep, int prec, const HopArgs &a, HopChoice c, cudaStream_t s)
{
    switch (rep * 3 + prec) {
    case 0: return launch_t<kRepFund, kF64>(ctx, g, a, c, s);
    case 1: return launch_t<kRepFund, kF32>(ctx, g, a, c, s);
    case 2: return launch_t<kRepFund, kF16>(ctx, g, a, c, s);
    case 3: return launch_t<kRepAdj, kF64>(ctx, g, a, c, s);
    case 4: return launch_t<kRepAdj, kF32>(ctx, g, a, c, s);
    case 5: return launch_t<kRepAdj, kF16>(ctx, g, a, c, s);
    case 6: return launch_t<kRepAdjMat, kF64>(ctx, g, a, c, s);
    case 7: return launch_t<kRepAdjMat, kF32>(ctx, g, a, c, s);
    case 8: return launch_t<kRepAdjMat, kF16>(ctx, g, a, c, s);
    }
    return set_error(ctx, HR_ERR_INVALID_ARG, "bad rep/prec");
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

hr_status launch_hop(hr_ctx *ctx, const Geom &g, int rep, int prec, const HopLaunch &L, cudaStream_t s)
{
    return dispatch(ctx, g, rep, prec, make_args(ctx, g, L), hop_choice(ctx, g, rep, prec), s);
}

hr_status launch_hop_with(hr_ctx *ctx, const Geom &g, int rep, int prec, const HopLaunch &L, HopChoice c,
                          cudaStream_t s)
{
    return dispatch(ctx, g, rep, prec, make_args(ctx, g, L), c, s);
}

bool hop_variant_available(int rep, int prec, int variant)
{
    (void)prec;
    return variant == kVarSimple || (variant >= kVarStaged && variant < kNumVariants && rep != HR_ADJ_MAT);
}

// Even-site operators from two hops each:
//   Mhat    : t_o = H_oe in;        out = A in - c H_eo t_o
//   Mhat^+  : t_o = H_oe g5 in;     out = A in - c g5 H_eo t_o
//   normal  : u = Mhat in (|u|^2 reduced with fin_schur), out = Mhat^+ u
// with A = 4 + m0 and c = 1 / (4 A).
hr_status apply_eo_op(hr_ctx *ctx, const Geom &g, double m0, int rep, int prec, int op, const void *gauge,
                      const void *in, void *out, void *work_odd, void *work_even, int fin_schur, const double *gate,
                      const double *done, cudaStream_t s)
{
    const double A = 4.0 + m0, c = 1.0 / (4.0 * A);
    hr_status st;
    HopLaunch L{};
    L.gauge = gauge;
    L.gate = gate;
    L.done = done;
    auto schur = [&](const void *src, void *dst, bool dag, int fin) -> hr_status {
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
        return launch_hop(ctx, g, rep, prec, h2, s);
    };
    switch (op) {
    case HR_OP_SCHUR: return schur(in, out, false, fin_schur);
    case HR_OP_SCHUR_DAG: return schur(in, out, true, fin_schur);
    case HR_OP_NORMAL:
        st = schur(in, work_even, false, fin_schur);
        if (st) return st;
        return schur(work_even, out, true, kFinNone);
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
    if (!gauge || !in || !out) return set_error(ctx, HR_ERR_INVALID_ARG, "null field pointer");
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
    if (!gauge || !in || !out) return set_error(ctx, HR_ERR_INVALID_ARG, "null field pointer");
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
