// hr_clover_leaf.cuh -- the link derivative of f = Re sum_y tr[C(y) Lam(y)]
// for fundamental SU(2) links, one link at a time, plaquette by plaquette
// (plain C++ as well as CUDA, HR_HD, so that the host can check it).
//
// With tr[C Lam] = (i/2) sum_{mu<nu} tr_c[F_mn K_mn] and F_mn(x) = (Q_mn(x) -
// Q_mn(x)^+) / 8, every plaquette P_w = a b c^+ d^+ of the (mu, nu) plane
// (a = U_mu(w), b = U_nu(w+mu), c = U_mu(w+nu), d = U_nu(w); corners w,
// w+mu, w+mu+nu, w+nu, traversed in that order) enters Q_mn at each of its
// four corners, as its cyclic rotation from that corner, so
//   f = Re (i/16) sum_{mu<nu} sum_w sum_corners tr[(R - R^+) K_corner],
// and sum_corners tr[R K] = tr[P with K_corner inserted at its corner].
// Rotating P to start at the varied link V (V = U for a, b; V = U^+ for c, d)
// and collecting the four insertions into Z (K) and Z' (K^+), the variation
// under dU = X U, X = i w.s/2, is Re (i/16) tr[X G] with
//   G = U Z + (U Z')^+          (V = U),      G = -(Z U^+ + (Z' U^+)^+)   (V = U^+),
// and the link's su(2) component a gains -Re tr(s_a G) / 32.  Each link lies
// on two plaquettes of each of the three planes that hold its direction.
// (The same sum as differentiating each leaf occurrence separately, with the
// four insertions of a plaquette sharing one staple product.)
#pragma once

#include "hr_eigh.cuh" // zd, HR_HD

namespace hr {

struct M2 {
    zd m[2][2];
};

HR_HD inline zd zd_add(zd a, zd b) { return {a.re + b.re, a.im + b.im}; }
HR_HD inline zd zd_mul(zd a, zd b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }

// A B with either factor optionally daggered
HR_HD inline M2 m2_mul(const M2 &A, bool da, const M2 &B, bool db)
{
    M2 C;
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) {
            zd s = {0.0, 0.0};
            for (int k = 0; k < 2; ++k) {
                const zd a = da ? zd{A.m[k][r].re, -A.m[k][r].im} : A.m[r][k];
                const zd b = db ? zd{B.m[c][k].re, -B.m[c][k].im} : B.m[k][c];
                s = zd_add(s, zd_mul(a, b));
            }
            C.m[r][c] = s;
        }
    return C;
}
HR_HD inline M2 m2_add(const M2 &A, const M2 &B)
{
    M2 C;
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) C.m[r][c] = zd_add(A.m[r][c], B.m[r][c]);
    return C;
}
HR_HD inline M2 m2_dag(const M2 &A)
{
    M2 C;
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) C.m[r][c] = {A.m[c][r].re, -A.m[c][r].im};
    return C;
}

// lattice with lexicographic sites ((x0 L1 + x1) L2 + x2) L3 + x3
struct LeafLattice {
    int d[4];
    HR_HD long long lex(const int (&x)[4]) const
    {
        return (((long long)x[0] * d[1] + x[1]) * d[2] + x[2]) * d[3] + x[3];
    }
    // x + s1 m1 + s2 m2 (periodic)
    HR_HD long long at(const int (&x)[4], int m1, int s1, int m2, int s2) const
    {
        int y[4] = {x[0], x[1], x[2], x[3]};
        y[m1] = ((y[m1] + s1) % d[m1] + d[m1]) % d[m1];
        y[m2] = ((y[m2] + s2) % d[m2] + d[m2]) % d[m2];
        return lex(y);
    }
};

// U_mu(x) from the canonical quaternion field double[4][V][4]
HR_HD inline M2 leaf_link(const double *can, long long V, int mu, long long x)
{
    const double *q = can + ((long long)mu * V + x) * 4;
    M2 U;
    U.m[0][0] = {q[0], q[3]};
    U.m[0][1] = {q[2], q[1]};
    U.m[1][0] = {-q[2], q[1]};
    U.m[1][1] = {q[0], -q[3]};
    return U;
}

// K_pl(x) (or its dagger) from the K field double[V][6][2][2][2]
HR_HD inline M2 leaf_k(const double *K, long long x, int pl, bool dag)
{
    const double *k = K + (x * 6 + pl) * 8;
    M2 M;
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) M.m[r][c] = {k[(r * 2 + c) * 2], k[(r * 2 + c) * 2 + 1]};
    return dag ? m2_dag(M) : M;
}

// G of one plaquette of the (mu, nu) plane (mu < nu, plane index pl) with
// lower corner w, for the varied link `which` (0: a, 1: b, 2: c, 3: d)
HR_HD inline M2 plaquette_g(const LeafLattice &L, const double *can, const double *K, int mu, int nu, int pl,
                            const int (&w)[4], int which)
{
    const long long V = (long long)L.d[0] * L.d[1] * L.d[2] * L.d[3];
    const long long s_w = L.lex(w), s_m = L.at(w, mu, 1, nu, 0), s_mn = L.at(w, mu, 1, nu, 1),
                    s_n = L.at(w, mu, 0, nu, 1);
    const M2 a = leaf_link(can, V, mu, s_w), b = leaf_link(can, V, nu, s_m), c = leaf_link(can, V, mu, s_n),
             d = leaf_link(can, V, nu, s_w);
    M2 G;
    for (int pass = 0; pass < 2; ++pass) {
        const bool kd = pass == 1; // Z' takes K^+
        const M2 Kw = leaf_k(K, s_w, pl, kd), Km = leaf_k(K, s_m, pl, kd), Kmn = leaf_k(K, s_mn, pl, kd),
                 Kn = leaf_k(K, s_n, pl, kd);
        M2 Z;
        if (which == 0) {
            // a (b c^+ d^+ Kw + Km b c^+ d^+ + b Kmn c^+ d^+ + b c^+ Kn d^+)
            const M2 cd = m2_mul(c, true, d, true), bc = m2_mul(b, false, c, true), S = m2_mul(b, false, cd, false);
            Z = m2_add(m2_add(m2_mul(S, false, Kw, false), m2_mul(Km, false, S, false)),
                       m2_add(m2_mul(m2_mul(b, false, Kmn, false), false, cd, false),
                              m2_mul(m2_mul(bc, false, Kn, false), false, d, true)));
        } else if (which == 1) {
            // b (Kmn c^+ d^+ a + c^+ Kn d^+ a + c^+ d^+ Kw a + c^+ d^+ a Km)
            const M2 cd = m2_mul(c, true, d, true), da = m2_mul(d, true, a, false), T = m2_mul(cd, false, a, false);
            Z = m2_add(m2_add(m2_mul(Kmn, false, T, false), m2_mul(m2_mul(c, true, Kn, false), false, da, false)),
                       m2_add(m2_mul(m2_mul(cd, false, Kw, false), false, a, false), m2_mul(T, false, Km, false)));
        } else if (which == 2) {
            // c^+ (Kn d^+ a b + d^+ Kw a b + d^+ a Km b + d^+ a b Kmn)
            const M2 ab = m2_mul(a, false, b, false), da = m2_mul(d, true, a, false), T = m2_mul(d, true, ab, false);
            Z = m2_add(m2_add(m2_mul(Kn, false, T, false), m2_mul(m2_mul(d, true, Kw, false), false, ab, false)),
                       m2_add(m2_mul(m2_mul(da, false, Km, false), false, b, false), m2_mul(T, false, Kmn, false)));
        } else {
            // d^+ (Kw a b c^+ + a Km b c^+ + a b Kmn c^+ + a b c^+ Kn)
            const M2 ab = m2_mul(a, false, b, false), bc = m2_mul(b, false, c, true), T = m2_mul(ab, false, c, true);
            Z = m2_add(m2_add(m2_mul(Kw, false, T, false), m2_mul(m2_mul(a, false, Km, false), false, bc, false)),
                       m2_add(m2_mul(m2_mul(ab, false, Kmn, false), false, c, true), m2_mul(T, false, Kn, false)));
        }
        const M2 &U = which == 0 ? a : which == 1 ? b : which == 2 ? c : d;
        // V = U: U Z and (U Z')^+;  V = U^+: Z U^+ and (Z' U^+)^+, with a minus sign
        const M2 t = which < 2 ? m2_mul(U, false, Z, false) : m2_mul(Z, false, U, true);
        const M2 term = kd ? m2_dag(t) : t;
        G = pass == 0 ? term : m2_add(G, term);
    }
    if (which >= 2)
        for (int r = 0; r < 2; ++r)
            for (int cc = 0; cc < 2; ++cc) G.m[r][cc] = {-G.m[r][cc].re, -G.m[r][cc].im};
    return G;
}

// out[a] = d f / d w_a for the link U_rho(z) (coordinates x of z)
HR_HD inline void leaf_force_link(const LeafLattice &L, const double *can, const double *K, int rho,
                                  const int (&x)[4], double (&out)[3])
{
    out[0] = out[1] = out[2] = 0.0;
    for (int pl = 0; pl < 6; ++pl) {
        // planes 01 02 03 12 13 23
        const int mu = pl < 3 ? 0 : (pl < 5 ? 1 : 2);
        const int nu = pl < 3 ? pl + 1 : (pl < 5 ? pl - 1 : 3);
        if (rho != mu && rho != nu) continue;
        for (int side = 0; side < 2; ++side) {
            // rho = mu: a of the plaquette at z, c of the plaquette at z - nu;
            // rho = nu: b of the plaquette at z - mu, d of the plaquette at z
            int w[4] = {x[0], x[1], x[2], x[3]};
            int which;
            if (rho == mu) {
                which = side == 0 ? 0 : 2;
                if (side == 1) w[nu] = (w[nu] - 1 + L.d[nu]) % L.d[nu];
            } else {
                which = side == 0 ? 1 : 3;
                if (side == 0) w[mu] = (w[mu] - 1 + L.d[mu]) % L.d[mu];
            }
            const M2 G = plaquette_g(L, can, K, mu, nu, pl, w, which);
            // -Re tr(s_a G) / 32
            out[0] -= (G.m[1][0].re + G.m[0][1].re) / 32.0;
            out[1] -= (G.m[1][0].im - G.m[0][1].im) / 32.0;
            out[2] -= (G.m[0][0].re - G.m[1][1].re) / 32.0;
        }
    }
}

} // namespace hr
