/*
 * hr_oracle.c -- plain FP64 CPU oracle for the Wilson-Dirac hot path.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load this code; the product path never does.  It shares no
 * code, header or table with the CUDA library.
 *
 * What it computes (the paper, arXiv:2411.18511, names the unimproved
 * Wilson-Dirac operator in Sec. 2.1 and Table 1, its even/odd split and
 * even-odd preconditioned form in Sec. 2.1, and inverters in Sec. 1, but
 * writes none of them down; the readings below are the textbook ones):
 *
 *   (D psi)(x) = (4+m0) psi(x)
 *              - 1/2 sum_mu [ (1-g_mu) U_mu(x) psi(x+mu)
 *                            + (1+g_mu) U_mu(x-mu)^+ psi(x-mu) ]
 *
 * with periodic boundaries, antiperiodic ones in the directions mu whose bit
 * (bc >> mu) & 1 is set, psi(x + L_mu mu-hat) = -psi(x), and twisted ones with
 * angle theta_mu, psi(x + L_mu mu-hat) = e^{i theta_mu} psi(x) (both together:
 * the product of the two factors).  A hop whose neighbour lies across the
 * boundary of direction mu picks up the factor that carries the stored value
 * over: e^{+i theta_mu} (times -1 if antiperiodic) stepping forward across it,
 * e^{-i theta_mu} (times -1) stepping backward.  theta may be NULL: no twist.  The chiral gamma basis
 *   g_0 = [[0, 1], [1, 0]],  g_k = [[0, -i s_k], [i s_k, 0]],  g5 = g0 g1 g2 g3,
 * SU(2) links U = a0 + i(a1 s1 + a2 s2 + a3 s3) in the fundamental
 * representation, and R_ab = 1/2 tr(s_a U s_b U^+) in the adjoint.  The hopping
 * term H is the bracket above (so D = (4+m0) - H/2).  Even-odd: the Schur
 * complement on even sites is  Mhat = (4+m0) - H_eo H_oe / (4 (4+m0)),  and
 * Mhat^+ = g5 Mhat g5.  CG is the Hestenes-Stiefel iteration on Mhat^+ Mhat.
 *
 * Everything is evaluated straight from these definitions: full 4x4 gamma
 * matrices, full colour matrices, no spin projection, no blocking.  Fields use
 * the canonical layouts:
 *   gauge  double [4][V][4]           quaternion per link
 *   links  complex [4][V][nc][nc]     expanded colour matrices
 *   spinor complex [V][4][nc]
 * with lexicographic site index ((x0*L1 + x1)*L2 + x2)*L3 + x3.
 *
 * Parity pins: free-field plane waves, flat connections, gamma5-hermiticity,
 * gauge covariance and dense brute force (tests/test_oracle_*.py).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

static cplx SIG[4][2][2];  /* SIG[0] = 1, SIG[1..3] = Pauli matrices */
static cplx GAM[5][4][4];  /* GAM[0..3] = gamma_mu, GAM[4] = gamma5 */
static int tables_ready = 0;

static void init_tables(void)
{
    if (tables_ready) return;
    memset(SIG, 0, sizeof SIG);
    memset(GAM, 0, sizeof GAM);
    SIG[0][0][0] = 1; SIG[0][1][1] = 1;
    SIG[1][0][1] = 1; SIG[1][1][0] = 1;
    SIG[2][0][1] = -I; SIG[2][1][0] = I;
    SIG[3][0][0] = 1; SIG[3][1][1] = -1;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            GAM[0][a][2 + b] = SIG[0][a][b];
            GAM[0][2 + a][b] = SIG[0][a][b];
            for (int k = 1; k <= 3; ++k) {
                GAM[k][a][2 + b] = -I * SIG[k][a][b];
                GAM[k][2 + a][b] = I * SIG[k][a][b];
            }
        }
    /* gamma5 = g0 g1 g2 g3 */
    cplx acc[4][4], tmp[4][4];
    memcpy(acc, GAM[0], sizeof acc);
    for (int k = 1; k <= 3; ++k) {
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) {
                cplx s = 0;
                for (int l = 0; l < 4; ++l) s += acc[i][l] * GAM[k][l][j];
                tmp[i][j] = s;
            }
        memcpy(acc, tmp, sizeof acc);
    }
    memcpy(GAM[4], acc, sizeof acc);
    tables_ready = 1;
}

/* ------------------------------------------------------------------ */
/* geometry                                                            */
/* ------------------------------------------------------------------ */

static long volume(const int *d) { return (long)d[0] * d[1] * d[2] * d[3]; }

static void coords(const int *d, long i, int x[4])
{
    x[3] = (int)(i % d[3]); i /= d[3];
    x[2] = (int)(i % d[2]); i /= d[2];
    x[1] = (int)(i % d[1]); i /= d[1];
    x[0] = (int)i;
}

static long lex(const int *d, const int x[4])
{
    return (((long)x[0] * d[1] + x[1]) * d[2] + x[2]) * d[3] + x[3];
}

/* site x + step * mu-hat with periodic wrap */
static long shift(const int *d, long i, int mu, int step)
{
    int x[4];
    coords(d, i, x);
    x[mu] = ((x[mu] + step) % d[mu] + d[mu]) % d[mu];
    return lex(d, x);
}

/* The boundary factor of the hop from site i to i + step * mu-hat (step = +-1):
 * 1 unless the step crosses the lattice's edge in direction mu; then -1 if mu
 * is antiperiodic (bit mu of bc), times e^{i step theta_mu} if th is given. */
static cplx wrap_phase(const int *d, int bc, const double *th, long i, int mu, int step)
{
    int x[4];
    coords(d, i, x);
    int y = x[mu] + step;
    if (y >= 0 && y < d[mu]) return 1.0;
    cplx f = ((bc >> mu) & 1) ? -1.0 : 1.0;
    if (th && th[mu] != 0.0) f *= cexp(I * (double)step * th[mu]);
    return f;
}

static int parity(const int *d, long i)
{
    int x[4];
    coords(d, i, x);
    return (x[0] + x[1] + x[2] + x[3]) & 1;
}

static int check_dims(const int *d)
{
    for (int mu = 0; mu < 4; ++mu)
        if (d[mu] < 2 || (d[mu] & 1)) return -1;
    return 0;
}

static int check_lat(const int *d, int bc, const double *th)
{
    if (check_dims(d) || bc < 0 || bc > 15) return -1;
    if (th)
        for (int mu = 0; mu < 4; ++mu)
            if (!isfinite(th[mu])) return -1;
    return 0;
}

/* ------------------------------------------------------------------ */
/* links                                                               */
/* ------------------------------------------------------------------ */

/* U = a0 * 1 + i * sum_k a_k s_k */
static void su2_from_quat(const double *a, cplx U[2][2])
{
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            cplx s = a[0] * SIG[0][i][j];
            for (int k = 1; k <= 3; ++k) s += I * a[k] * SIG[k][i][j];
            U[i][j] = s;
        }
}

static void mat2_mul(const cplx A[2][2], const cplx B[2][2], cplx C[2][2])
{
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) C[i][j] = A[i][0] * B[0][j] + A[i][1] * B[1][j];
}

static void mat2_dag(const cplx A[2][2], cplx B[2][2])
{
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) B[i][j] = conj(A[j][i]);
}

/* adjoint representation R_ab = 1/2 tr(s_a U s_b U^+), a, b = 1..3 */
static void adj_from_quat(const double *q, double R[3][3])
{
    cplx U[2][2], Ud[2][2], t1[2][2], t2[2][2], t3[2][2];
    su2_from_quat(q, U);
    mat2_dag(U, Ud);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            mat2_mul(SIG[a + 1], U, t1);
            mat2_mul(t1, SIG[b + 1], t2);
            mat2_mul(t2, Ud, t3);
            R[a][b] = 0.5 * creal(t3[0][0] + t3[1][1]);
        }
}

/* Expand quaternion links to colour matrices: L[mu][V][nc][nc] complex. */
int or_expand_links(const int *d, int nc, const double *q, double *Lout)
{
    init_tables();
    if (check_dims(d) || (nc != 2 && nc != 3)) return -1;
    long V = volume(d);
    cplx *L = (cplx *)Lout;
    for (long l = 0; l < 4 * V; ++l) {
        cplx *m = L + l * nc * nc;
        if (nc == 2) {
            cplx U[2][2];
            su2_from_quat(q + 4 * l, U);
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j) m[i * 2 + j] = U[i][j];
        } else {
            double R[3][3];
            adj_from_quat(q + 4 * l, R);
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) m[i * 3 + j] = R[i][j];
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* hopping term                                                         */
/* ------------------------------------------------------------------ */

/* out[s][c] = (H psi)(x) at one site, straight from the definition */
static void hop_site(const int *d, int bc, const double *th, int nc, const cplx *L, const cplx *psi, long x,
                     cplx *out)
{
    long V = volume(d);
    int ns = 4 * nc;
    for (int k = 0; k < ns; ++k) out[k] = 0;
    for (int mu = 0; mu < 4; ++mu) {
        long xf = shift(d, x, mu, +1), xb = shift(d, x, mu, -1);
        /* psi(x +- mu) across the boundary is the stored value times its factor */
        cplx sgf = wrap_phase(d, bc, th, x, mu, +1), sgb = wrap_phase(d, bc, th, x, mu, -1);
        const cplx *Uf = L + ((long)mu * V + x) * nc * nc;
        const cplx *Ub = L + ((long)mu * V + xb) * nc * nc;
        const cplx *pf = psi + xf * ns, *pb = psi + xb * ns;
        cplx tf[4][3], tb[4][3];
        for (int s = 0; s < 4; ++s)
            for (int c = 0; c < nc; ++c) {
                cplx sf = 0, sb = 0;
                for (int e = 0; e < nc; ++e) {
                    sf += Uf[c * nc + e] * pf[s * nc + e];        /* U_mu(x) psi(x+mu)     */
                    sb += conj(Ub[e * nc + c]) * pb[s * nc + e];  /* U_mu(x-mu)^+ psi(x-mu) */
                }
                tf[s][c] = sgf * sf;
                tb[s][c] = sgb * sb;
            }
        for (int s = 0; s < 4; ++s)
            for (int c = 0; c < nc; ++c) {
                cplx acc = 0;
                for (int t = 0; t < 4; ++t) {
                    cplx one = (s == t) ? 1.0 : 0.0;
                    acc += (one - GAM[mu][s][t]) * tf[t][c];
                    acc += (one + GAM[mu][s][t]) * tb[t][c];
                }
                out[s * nc + c] += acc;
            }
    }
}

/* out(x) = (H psi)(x) for every x of the given parity (-1: every site).
 * Sites of the other parity in out are left untouched. */
int or_hop(const int *d, int bc, const double *th, int nc, const double *Lr, int par, const double *psir,
           double *outr)
{
    init_tables();
    if (check_lat(d, bc, th) || (nc != 2 && nc != 3)) return -1;
    long V = volume(d);
    const cplx *L = (const cplx *)Lr, *psi = (const cplx *)psir;
    cplx *out = (cplx *)outr;
    int ns = 4 * nc;
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; ++x) {
        if (par >= 0 && parity(d, x) != par) continue;
        hop_site(d, bc, th, nc, L, psi, x, out + x * ns);
    }
    return 0;
}

/* out[j] = (H psi)(sites[j]); out is [n][4][nc] */
int or_hop_sites(const int *d, int bc, const double *th, int nc, const double *Lr, const long *sites, long n,
                 const double *psir, double *outr)
{
    init_tables();
    if (check_lat(d, bc, th) || (nc != 2 && nc != 3)) return -1;
    long V = volume(d);
    for (long j = 0; j < n; ++j)
        if (sites[j] < 0 || sites[j] >= V) return -2;
    const cplx *L = (const cplx *)Lr, *psi = (const cplx *)psir;
    cplx *out = (cplx *)outr;
#pragma omp parallel for schedule(static)
    for (long j = 0; j < n; ++j) hop_site(d, bc, th, nc, L, psi, sites[j], out + j * 4 * nc);
    return 0;
}

/* full operator: out = (4+m0) psi - 1/2 H psi */
int or_dirac(const int *d, int bc, const double *th, int nc, const double *Lr, double m0, const double *psir,
             double *outr)
{
    int rc = or_hop(d, bc, th, nc, Lr, -1, psir, outr);
    if (rc) return rc;
    long n = volume(d) * 4 * nc;
    const cplx *psi = (const cplx *)psir;
    cplx *out = (cplx *)outr;
    for (long k = 0; k < n; ++k) out[k] = (4.0 + m0) * psi[k] - 0.5 * out[k];
    return 0;
}

static void apply_g5(int nc, long V, cplx *v)
{
    /* gamma5 is diagonal in the chiral basis: multiply spin s by GAM[4][s][s] */
    for (long x = 0; x < V; ++x)
        for (int s = 0; s < 4; ++s)
            for (int c = 0; c < nc; ++c) v[(x * 4 + s) * nc + c] *= GAM[4][s][s];
}

/* Mhat psi on even sites (dagger = 0) or Mhat^+ psi = g5 Mhat g5 psi (dagger = 1).
 * psi, out: full-lattice arrays; only even sites of psi are read, odd sites of
 * out are set to zero. */
int or_schur(const int *d, int bc, const double *th, int nc, const double *Lr, double m0, int dagger,
             const double *psir, double *outr)
{
    init_tables();
    if (check_lat(d, bc, th) || (nc != 2 && nc != 3)) return -1;
    long V = volume(d), n = V * 4 * nc;
    double A = 4.0 + m0;
    cplx *in = calloc(n, sizeof(cplx)), *t = calloc(n, sizeof(cplx));
    cplx *u = calloc(n, sizeof(cplx));
    if (!in || !t || !u) { free(in); free(t); free(u); return -3; }
    const cplx *psi = (const cplx *)psir;
    for (long x = 0; x < V; ++x)
        if (parity(d, x) == 0) memcpy(in + x * 4 * nc, psi + x * 4 * nc, 4 * nc * sizeof(cplx));
    if (dagger) apply_g5(nc, V, in);
    or_hop(d, bc, th, nc, Lr, 1, (const double *)in, (double *)t);  /* t_o = H_oe in_e   */
    or_hop(d, bc, th, nc, Lr, 0, (const double *)t, (double *)u);   /* u_e = H_eo t_o    */
    cplx *out = (cplx *)outr;
    for (long x = 0; x < V; ++x) {
        cplx *o = out + x * 4 * nc;
        if (parity(d, x) != 0) {
            for (int k = 0; k < 4 * nc; ++k) o[k] = 0;
            continue;
        }
        for (int k = 0; k < 4 * nc; ++k) o[k] = A * in[x * 4 * nc + k] - u[x * 4 * nc + k] / (4.0 * A);
    }
    if (dagger) apply_g5(nc, V, out);
    free(in); free(t); free(u);
    return 0;
}

/* out = Mhat^+ Mhat psi (even sites) */
int or_normal(const int *d, int bc, const double *th, int nc, const double *Lr, double m0, const double *psir,
              double *outr)
{
    long n = volume(d) * 4 * nc;
    double *tmp = calloc(2 * n, sizeof(double));
    if (!tmp) return -3;
    int rc = or_schur(d, bc, th, nc, Lr, m0, 0, psir, tmp);
    if (!rc) rc = or_schur(d, bc, th, nc, Lr, m0, 1, tmp, outr);
    free(tmp);
    return rc;
}

static double dotre(long n, const cplx *a, const cplx *b)
{
    double s = 0;
    for (long k = 0; k < n; ++k) s += creal(conj(a[k]) * b[k]);
    return s;
}

/* Hestenes-Stiefel CG on Mhat^+ Mhat x = b (even sites), x0 = 0.
 * Stops when the iterated residual satisfies |r| <= tol |b|; then returns the
 * true relative residual |b - A x| / |b| recomputed from x. */
int or_cg(const int *d, int bc, const double *th, int nc, const double *Lr, double m0, const double *br, double *xr,
          double tol, int maxiter, int *iters, double *true_rel)
{
    init_tables();
    if (check_lat(d, bc, th) || (nc != 2 && nc != 3)) return -1;
    long n = volume(d) * 4 * nc;
    const cplx *b = (const cplx *)br;
    cplx *x = (cplx *)xr;
    cplx *r = malloc(n * sizeof(cplx)), *p = malloc(n * sizeof(cplx)), *q = malloc(n * sizeof(cplx));
    if (!r || !p || !q) { free(r); free(p); free(q); return -3; }
    for (long k = 0; k < n; ++k) { x[k] = 0; r[k] = b[k]; p[k] = b[k]; }
    double bb = dotre(n, b, b), rr = bb;
    int it = 0;
    while (it < maxiter && sqrt(rr / bb) > tol) {
        or_normal(d, bc, th, nc, Lr, m0, (const double *)p, (double *)q);
        double alpha = rr / dotre(n, p, q);
        for (long k = 0; k < n; ++k) { x[k] += alpha * p[k]; r[k] -= alpha * q[k]; }
        double rr_new = dotre(n, r, r);
        double beta = rr_new / rr;
        for (long k = 0; k < n; ++k) p[k] = r[k] + beta * p[k];
        rr = rr_new;
        ++it;
    }
    or_normal(d, bc, th, nc, Lr, m0, (const double *)x, (double *)q);
    for (long k = 0; k < n; ++k) r[k] = b[k] - q[k];
    *true_rel = sqrt(dotre(n, r, r) / bb);
    *iters = it;
    free(r); free(p); free(q);
    return (sqrt(rr / bb) <= tol) ? 0 : 1;
}

/* ------------------------------------------------------------------ */
/* link derivatives of f = Re <a, H b>  (fundamental representation)    */
/* ------------------------------------------------------------------ */

/* Under U_mu(x) -> exp(eps X) U_mu(x), X = i sum_a w_a s_a / 2, the two terms of
 * H containing the link give
 *   df/deps = Re tr[ X (Q1 - Q2) ],
 *   Q1 = sum_s (U b(x+mu))_s [((1-g_mu) a(x))_s]^+,
 *   Q2 = sum_s b(x)_s [(U (1+g_mu) a(x+mu))_s]^+.
 * F[mu][x][a-1] = d f / d w_a = Re tr[(i s_a / 2)(Q1 - Q2)], a = 1..3.
 * Across the boundary the hop x -> x+mu carries its factor f (wrap_phase, step
 * +1) and the hop x+mu -> x its factor fb (step -1): the two terms become
 * f Q1 and fb Q2 (for antiperiodic directions both are -1). */
int or_force(const int *d, int bc, const double *th, const double *Lr, const double *ar, const double *br,
             double *F)
{
    init_tables();
    if (check_lat(d, bc, th)) return -1;
    long V = volume(d);
    const cplx *L = (const cplx *)Lr, *a = (const cplx *)ar, *b = (const cplx *)br;
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; ++x) {
        for (int mu = 0; mu < 4; ++mu) {
            long xf = shift(d, x, mu, +1);
            const cplx *U = L + ((long)mu * V + x) * 4;
            cplx pa[4][2], pa2[4][2], Ub[4][2], Upa[4][2];
            for (int s = 0; s < 4; ++s)
                for (int c = 0; c < 2; ++c) {
                    cplx s1 = 0, s2 = 0;
                    for (int t = 0; t < 4; ++t) {
                        cplx one = (s == t) ? 1.0 : 0.0;
                        s1 += (one - GAM[mu][s][t]) * a[(x * 4 + t) * 2 + c];
                        s2 += (one + GAM[mu][s][t]) * a[(xf * 4 + t) * 2 + c];
                    }
                    pa[s][c] = s1;
                    pa2[s][c] = s2;
                }
            for (int s = 0; s < 4; ++s)
                for (int c = 0; c < 2; ++c) {
                    Ub[s][c] = U[c * 2 + 0] * b[(xf * 4 + s) * 2 + 0] + U[c * 2 + 1] * b[(xf * 4 + s) * 2 + 1];
                    Upa[s][c] = U[c * 2 + 0] * pa2[s][0] + U[c * 2 + 1] * pa2[s][1];
                }
            cplx f = wrap_phase(d, bc, th, x, mu, +1), fb = wrap_phase(d, bc, th, xf, mu, -1);
            cplx Q[2][2];
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j) {
                    cplx q1 = 0, q2 = 0;
                    for (int sp = 0; sp < 4; ++sp) {
                        q1 += Ub[sp][i] * conj(pa[sp][j]);
                        q2 += b[(x * 4 + sp) * 2 + i] * conj(Upa[sp][j]);
                    }
                    Q[i][j] = f * q1 - fb * q2;
                }
            for (int k = 1; k <= 3; ++k) {
                cplx tr = 0;
                for (int i = 0; i < 2; ++i)
                    for (int j = 0; j < 2; ++j) tr += 0.5 * I * SIG[k][i][j] * Q[j][i];
                F[((long)mu * V + x) * 3 + (k - 1)] = creal(tr);
            }
        }
    }
    return 0;
}

/* G[mu][x][k] = d Re<a, H b> / d a_k for the link quaternion of U_mu(x),
 * U = sum_k a_k E_k with E_0 = 1, E_k = i s_k:
 *   = Re[f a(x)^+ (1-g_mu) E_k b(x+mu)] + Re[fb a(x+mu)^+ (1+g_mu) E_k^+ b(x)],
 * f and fb the boundary factors of the two hops (1 off the boundary), as for
 * the force. */
int or_link_grad(const int *d, int bc, const double *th, const double *ar, const double *br, double *G)
{
    init_tables();
    if (check_lat(d, bc, th)) return -1;
    long V = volume(d);
    const cplx *a = (const cplx *)ar, *b = (const cplx *)br;
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; ++x) {
        for (int mu = 0; mu < 4; ++mu) {
            long xf = shift(d, x, mu, +1);
            cplx f = wrap_phase(d, bc, th, x, mu, +1), fb = wrap_phase(d, bc, th, xf, mu, -1);
            for (int k = 0; k < 4; ++k) {
                cplx E[2][2], Ed[2][2];
                for (int i = 0; i < 2; ++i)
                    for (int j = 0; j < 2; ++j) E[i][j] = (k == 0) ? SIG[0][i][j] : I * SIG[k][i][j];
                mat2_dag(E, Ed);
                cplx acc = 0;
                for (int s = 0; s < 4; ++s)
                    for (int t = 0; t < 4; ++t) {
                        cplx one = (s == t) ? 1.0 : 0.0;
                        cplx gm = one - GAM[mu][s][t], gp = one + GAM[mu][s][t];
                        for (int i = 0; i < 2; ++i)
                            for (int j = 0; j < 2; ++j) {
                                acc += f * conj(a[(x * 4 + s) * 2 + i]) * gm * E[i][j] * b[(xf * 4 + t) * 2 + j];
                                acc += fb * conj(a[(xf * 4 + s) * 2 + i]) * gp * Ed[i][j] * b[(x * 4 + t) * 2 + j];
                            }
                    }
                G[((long)mu * V + x) * 4 + k] = creal(acc);
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* misc                                                                 */
/* ------------------------------------------------------------------ */

/* <P> = 1/(6V) sum_{x, mu<nu} 1/2 Re tr U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+ */
int or_plaquette(const int *d, const double *q, double *P)
{
    init_tables();
    if (check_dims(d)) return -1;
    long V = volume(d);
    double acc = 0;
    for (long x = 0; x < V; ++x)
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = mu + 1; nu < 4; ++nu) {
                cplx U1[2][2], U2[2][2], U3[2][2], U4[2][2], U3d[2][2], U4d[2][2], t1[2][2], t2[2][2], t3[2][2];
                su2_from_quat(q + ((long)mu * V + x) * 4, U1);
                su2_from_quat(q + ((long)nu * V + shift(d, x, mu, 1)) * 4, U2);
                su2_from_quat(q + ((long)mu * V + shift(d, x, nu, 1)) * 4, U3);
                su2_from_quat(q + ((long)nu * V + x) * 4, U4);
                mat2_dag(U3, U3d);
                mat2_dag(U4, U4d);
                mat2_mul(U1, U2, t1);
                mat2_mul(t1, U3d, t2);
                mat2_mul(t2, U4d, t3);
                acc += 0.5 * creal(t3[0][0] + t3[1][1]);
            }
    *P = acc / (6.0 * V);
    return 0;
}

/* gamma matrix mu = 0..3, or gamma5 for mu = 4, as a 4x4 complex array */
int or_gamma(int mu, double *out)
{
    init_tables();
    if (mu < 0 || mu > 4) return -1;
    memcpy(out, GAM[mu], sizeof(GAM[mu]));
    return 0;
}

int or_adjoint_link(const double *q, double *R)
{
    init_tables();
    double M[3][3];
    adj_from_quat(q, M);
    memcpy(R, M, sizeof M);
    return 0;
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* threads for the following parallel loops (n >= 1); returns the previous count */
int or_set_num_threads(int n)
{
    int prev = or_num_threads();
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
    return prev;
}
