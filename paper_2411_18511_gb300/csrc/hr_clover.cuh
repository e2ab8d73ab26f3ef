// hr_clover.cuh -- layout of the packed clover field and its site product,
// shared by the hop epilogue (every kernel family) and the clover kernels.
//
// The clover (Sheikholeslami-Wohlert) and exponential-clover terms of
// arXiv:2411.18511 Sec. 2.2 are site-diagonal: A(x) = (4 + m0) + c_sw C(x), or
// (4 + m0) exp(c_sw C(x) / (4 + m0)), with C = (i/4) sum_{mu != nu} s_mn F_mn
// Hermitian and commuting with g5.  In the chiral basis A is two Hermitian
// n x n blocks, n = 2 NC: block 0 acts on spins 0, 1 and block 1 on spins
// 2, 3, on the index k = (spin - 2 b) * NC + colour.
//
// Packed field: four half-fields of V/2 sites each, in this order
//   [A on even sites | A on odd sites | A^-1 on even sites | A^-1 on odd sites]
// each padded to 256 bytes.  Per site the two blocks follow one another, each
// as n^2 reals: the n diagonal entries, then the upper triangle (r < c, row
// by row) as (re, im).  FP64 reals are double-float pairs (hi, lo): two reals
// per 16-byte vector; FP32: four.  Vectors of 32 consecutive sites interleave
// (AoSoA), as in the spinor layout, so a warp reads 512 contiguous bytes.
#pragma once

#include "hr_internal.cuh"

namespace hr {

template <int NC, int CP> struct CloverLayout {
    static constexpr int N = 2 * NC;         // block size
    static constexpr int NREAL = 2 * N * N;  // both blocks
    static constexpr int PER_VEC = CP == kF64 ? 2 : 4;
    static constexpr int NVEC = NREAL / PER_VEC;
    static_assert(NREAL % PER_VEC == 0, "whole vectors per site");
    static size_t half_bytes(int nblk) { return ((size_t)nblk * 32 * NVEC * 16 + 255) & ~(size_t)255; }
};

// clover storage precision of an operator precision: FP32 for FP32 and FP16 operators
__host__ __device__ constexpr int clover_prec(int prec) { return prec == kF64 ? kF64 : kF32; }

// real r of site i in a half-field
template <int NC, int CP, class T> struct CloverReader {
    using L = CloverLayout<NC, CP>;
    const float4 *base;
    int i;
    float4 w;
    int loaded = -1;
    __device__ __forceinline__ CloverReader(const void *half, int site) : base((const float4 *)half), i(site) {}
    __device__ __forceinline__ T get(int r)
    {
        const int v = r / L::PER_VEC, e = r % L::PER_VEC;
        if (v != loaded) {
            w = __ldg(base + ((size_t)(i >> 5) * L::NVEC + v) * 32 + (i & 31));
            loaded = v;
        }
        if constexpr (CP == kF64) {
            if constexpr (std::is_same<T, dd>::value) return e == 0 ? dd(w.x, w.y) : dd(w.z, w.w);
            else return e == 0 ? w.x + w.y : w.z + w.w;
        } else {
            return e == 0 ? w.x : e == 1 ? w.y : e == 2 ? w.z : w.w;
        }
    }
};

// v = A(x) v at site i (both blocks), A from the half-field `half`
template <int CP, class T, int NC>
__device__ __forceinline__ void clover_apply(const void *half, int i, cpx<T> (&v)[4][NC])
{
    constexpr int N = 2 * NC;
    CloverReader<NC, CP, T> rd(half, i);
    int r = 0;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        cpx<T> x[N], y[N];
#pragma unroll
        for (int k = 0; k < N; ++k) x[k] = v[2 * b + k / NC][k % NC];
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const T d = rd.get(r++);
            y[k] = {d * x[k].re, d * x[k].im};
        }
#pragma unroll
        for (int p = 0; p < N; ++p)
#pragma unroll
            for (int q = p + 1; q < N; ++q) {
                const T are = rd.get(r++), aim = rd.get(r++);
                // y_p += a x_q, y_q += conj(a) x_p
                y[p].re = y[p].re + (are * x[q].re - aim * x[q].im);
                y[p].im = y[p].im + (are * x[q].im + aim * x[q].re);
                y[q].re = y[q].re + (are * x[p].re + aim * x[p].im);
                y[q].im = y[q].im + (are * x[p].im - aim * x[p].re);
            }
#pragma unroll
        for (int k = 0; k < N; ++k) v[2 * b + k / NC][k % NC] = y[k];
    }
}

} // namespace hr
