/*
 * hirep_gb300.h -- C ABI of libhirep_gb300.so, the even-odd Wilson-Dirac hot
 * path for SU(2) gauge links on one NVIDIA GB300 (sm_103a).
 *
 * What the library computes.  arXiv:2411.18511 ("Scaling SU(2) to 1000 GPUs
 * using HiRep") measures the unimproved Wilson-Dirac operator (Sec. 2.1,
 * Table 1), its even/odd split and its even-odd preconditioned form "used
 * mainly in the HMC" (Sec. 2.1), for SU(2) with fermions in the fundamental and
 * higher representations (Sec. 1), inside the code's inverters (Sec. 1).  The
 * paper prints no formula; this library implements the textbook operator
 *
 *   (D psi)(x) = (4+m0) psi(x) - 1/2 (H psi)(x),
 *   (H psi)(x) = sum_mu (1-g_mu) U_mu(x) psi(x+mu) + (1+g_mu) U_mu(x-mu)^+ psi(x-mu),
 *
 * periodic in all four directions, chiral gamma basis
 *   g_0 = [[0,1],[1,0]], g_k = [[0,-i s_k],[i s_k,0]], g5 = g0 g1 g2 g3 = diag(-1,-1,1,1),
 * kappa = 1/(8 + 2 m0), and on even sites the Schur complement
 *
 *   Mhat = (4+m0) - H_eo H_oe / (4 (4+m0)),   Mhat^+ = g5 Mhat g5.
 *
 * Representations: HR_FUND (SU(2) fundamental, 2 complex colours) and the
 * adjoint (3 colours, real links R_ab = 1/2 tr(s_a U s_b U^+)).
 *
 * Conventions common to every call
 * --------------------------------
 * - Lattice extents (T, L1, L2, L3), each even and >= 2.  Site x = (x0..x3)
 *   has lexicographic index ((x0*L1 + x1)*L2 + x2)*L3 + x3 and parity
 *   (x0+x1+x2+x3) mod 2 (even = 0).  V = T*L1*L2*L3, V_h = V/2.
 * - Canonical ("user") layouts, FP64:
 *     gauge  double[4][V][4]      link U_mu(x) as quaternion (a0,a1,a2,a3),
 *                                 U = a0 + i(a1 s1 + a2 s2 + a3 s3)
 *     spinor double[V][4][nc][2]  site, spin, colour, (re, im)
 * - Packed layouts are opaque device buffers sized by hr_*_packed_bytes; the
 *   kernels read and write packed data only.  A packed spinor of one parity
 *   holds V_h sites; a "full" packed spinor is the even half followed by the
 *   odd half.  Packed buffers and work buffers must be 16-byte aligned,
 *   canonical buffers 8-byte aligned (cudaMalloc and torch allocations are);
 *   a null or misaligned buffer returns HR_ERR_INVALID_ARG before any launch.
 * - Ownership: the caller owns every buffer (device pointers, allocated by
 *   the caller) and the stream.  No hot call allocates memory.  Work buffers
 *   are passed in, sized by hr_workspace_bytes.  Calls are asynchronous on
 *   the given stream unless stated otherwise.
 * - A context's device scratch (reduction partials, solver scalars) is shared
 *   by the calls made with it: calls on one context must not overlap in time
 *   (use one stream per context, or one context per stream).
 * - Errors: every call returns hr_status; argument errors are detected on the
 *   host before anything is launched; hr_last_error() gives a message.
 */
#ifndef HIREP_GB300_H
#define HIREP_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *hr_stream; /* cudaStream_t; NULL = legacy default stream */

typedef enum {
    HR_OK = 0,
    HR_ERR_INVALID_ARG = 1,   /* bad pointer, size, enum or extent              */
    HR_ERR_UNSUPPORTED = 2,   /* valid but not implemented (odd extent, combo)  */
    HR_ERR_CUDA = 3,          /* a CUDA runtime call failed                     */
    HR_ERR_NOT_CONVERGED = 4, /* solver hit maxiter; x holds the last iterate   */
    HR_ERR_NUMERIC = 5,       /* NaN or Inf met in a residual                   */
    HR_ERR_TIMEOUT = 6,       /* a bounded device wait gave up                  */
    HR_ERR_WORKSPACE = 7      /* workspace too small                            */
} hr_status;

typedef enum {
    HR_FUND = 0,    /* fundamental: 2 complex colours, links stored as quaternions        */
    HR_ADJ = 1,     /* adjoint: 3 colours, links stored as quaternions, R(U) rebuilt in registers */
    HR_ADJ_MAT = 2  /* adjoint: as HR_ADJ but links stored as 3x3 real matrices R(U)    */
} hr_rep;

typedef enum {
    HR_F64 = 0, /* FP64 class: each real packed as an unevaluated pair of floats (hi + lo,
                   48 significant bits, about 3.6e-15 relative) and computed with error-free
                   float transformations; the canonical buffers stay IEEE binary64.  Full
                   precision for magnitudes 2^-102 (2e-31) .. 2^120 (1.3e36): see hr_ctx_status */
    HR_F32 = 1, /* FP32 storage and arithmetic                                            */
    HR_F16 = 2  /* binary16 storage (spinors scaled by a per-site FP32 max-abs), FP32 arithmetic */
} hr_prec;

typedef enum { HR_EVEN = 0, HR_ODD = 1, HR_FULL = 2 } hr_parity;

typedef enum {
    HR_OP_HOP = 0,       /* out_p = D_{p,1-p} in = -1/2 H_{p,1-p} in  (in on parity 1-p) */
    HR_OP_SCHUR = 1,     /* out_e = Mhat in_e           (out_parity must be HR_EVEN)   */
    HR_OP_SCHUR_DAG = 2, /* out_e = Mhat^+ in_e                                       */
    HR_OP_NORMAL = 3     /* out_e = Mhat^+ Mhat in_e                                  */
} hr_op;

/* A lattice: extents (T, L1, L2, L3), each even and >= 2, and its fermion
 * boundary conditions.  Bit mu of bc (HR_BC_ANTIPERIODIC(mu), mu = 0 is time)
 * makes direction mu antiperiodic, psi(x + L_mu mu-hat) = -psi(x); bc = 0 is
 * periodic in all four directions.  (The paper, arXiv:2411.18511, states no
 * boundary condition; antiperiodic time is the usual choice for fermions.)
 *
 * Where bc acts: hr_gauge_pack folds the sign into the packed links of the
 * last slice x_mu = L_mu - 1 of each antiperiodic direction (every hop that
 * crosses the boundary uses one of those links), so a packed gauge field
 * carries its boundary conditions into every operator, solver and force
 * applied with it.  hr_link_grad, which takes no gauge field, applies the
 * sign itself.  Other calls ignore bc.  bc outside [0, 15]: HR_ERR_INVALID_ARG.
 *
 * theta[mu] twists direction mu by a U(1) phase, psi(x + L_mu mu-hat) =
 * e^{i theta_mu} psi(x) (times -1 if bit mu of bc is set as well): a hop that
 * crosses that boundary forward picks up e^{+i theta_mu}, backward
 * e^{-i theta_mu}.  theta = 0 in all four directions (a zero-initialised
 * struct) is the untwisted lattice, and theta_mu = pi is the antiperiodic
 * sign.  The twist is not folded into the packed links (a phased SU(2) link
 * is no quaternion): the hop kernels apply it, so every call that applies the
 * operator to a twisted lattice -- hr_dirac_apply / _eo (and their clover
 * forms), the solvers, hr_force, hr_link_grad, hr_hmc_trajectory -- takes the
 * same lattice.  Those calls run a separate, untuned hop kernel for twisted
 * lattices; hr_cg_solve_batch returns HR_ERR_UNSUPPORTED for them.  A
 * non-finite angle: HR_ERR_INVALID_ARG. */
typedef struct {
    int dims[4];
    int bc;
    double theta[4];
} hr_lattice;
#define HR_BC_ANTIPERIODIC(mu) (1 << (mu))

typedef struct hr_ctx hr_ctx;

/* ---------------------------------------------------------------------- */
/* context                                                                  */
/* ---------------------------------------------------------------------- */

/* Create a context on CUDA device `device`: allocates its small device
 * scratch (reduction partials, solver scalars, status word; < 4 MB) once.
 * *ctx receives the handle; HR_ERR_CUDA if the device cannot be used. */
hr_status hr_ctx_create(hr_ctx **ctx, int device);
hr_status hr_ctx_destroy(hr_ctx *ctx);
/* Message of the last failed call on this context ("" if none). Never NULL. */
const char *hr_last_error(const hr_ctx *ctx);

/* The value-range status of the fields packed with this context since the
 * last check.  The packed layouts hold reals in the float exponent range (the
 * FP64 class as pairs of floats), so hr_gauge_pack and hr_spinor_pack flag,
 * on the device and without stopping, every canonical value that is NaN or
 * Inf or exceeds 2^120 = 1.3e36 in magnitude (beyond that an operator's sums
 * could overflow).  This call synchronises the stream, clears the flags and
 * returns HR_ERR_NUMERIC (a NaN or Inf was packed), HR_ERR_UNSUPPORTED (a value
 * above 2^120) or HR_OK.  The solvers (hr_cg_solve, hr_cg_solve_clover,
 * hr_solve_full, hr_cg_solve_batch, hr_hmc_trajectory) make the same check
 * before they start and return the same codes.  Small magnitudes are not
 * flagged: a pair keeps 48 bits down to 2^-102 (its low float stays normal)
 * and loses them gradually below, which matters only relative to the field's
 * largest component (the solvers check that, see hr_cg_solve). */
hr_status hr_ctx_status(hr_ctx *ctx, hr_stream stream);
/* Library version string. */
const char *hr_version(void);

/* m0 = 1/(2 kappa) - 4, i.e. kappa = 1/(8 + 2 m0). */
double hr_kappa_to_m0(double kappa);
double hr_m0_to_kappa(double m0);

/* ---------------------------------------------------------------------- */
/* sizes and layout conversion                                             */
/* ---------------------------------------------------------------------- */

/* Bytes of a packed gauge field (all 4V links, both parities); 0 if invalid. */
size_t hr_gauge_packed_bytes(hr_lattice lat, hr_rep rep, hr_prec prec);
/* Bytes of a packed spinor field: one parity (V_h sites) times n_rhs
 * right-hand sides (parity = HR_EVEN/HR_ODD), or both halves (HR_FULL). */
size_t hr_spinor_packed_bytes(hr_lattice lat, hr_rep rep, hr_prec prec, hr_parity parity, int n_rhs);

/* canonical gauge (device, double[4][V][4]) -> packed (device); values out of
 * range are flagged (hr_ctx_status).  For HR_ADJ_MAT
 * the 3x3 adjoint matrices are built on the GPU from the quaternions.  The
 * boundary sign of lat.bc is folded in: HR_FUND stores -q on the boundary
 * slice; HR_ADJ stores the representative of +-q whose q0 has its sign bit
 * clear, and sets that bit on the boundary slice (R(q) = R(-q), so the sign
 * bit is free to carry the factor -1 that the kernels apply to R); HR_ADJ_MAT
 * stores -R there.  A packed gauge field is therefore specific to its rep. */
hr_status hr_gauge_pack(hr_ctx *ctx, hr_lattice lat, hr_rep rep, hr_prec prec,
                        const double *canonical, void *packed, hr_stream stream);

/* canonical spinor(s) (device, double[n_rhs][V][4][nc][2]) -> packed sites of
 * `parity` (HR_FULL: both halves).  n_rhs > 1 gives the multi-RHS layout.
 * NaN, Inf and magnitudes above 2^120 are flagged (hr_ctx_status). */
hr_status hr_spinor_pack(hr_ctx *ctx, hr_lattice lat, hr_rep rep, hr_prec prec, hr_parity parity,
                         int n_rhs, const double *canonical, void *packed, hr_stream stream);
/* packed -> canonical; writes only the sites of `parity` (all for HR_FULL). */
hr_status hr_spinor_unpack(hr_ctx *ctx, hr_lattice lat, hr_rep rep, hr_prec prec, hr_parity parity,
                           int n_rhs, const void *packed, double *canonical, hr_stream stream);

/* ---------------------------------------------------------------------- */
/* operators                                                               */
/* ---------------------------------------------------------------------- */

/* Work bytes needed by hr_dirac_eo (op) / hr_dirac_apply for n_rhs vectors. */
size_t hr_dirac_workspace_bytes(hr_lattice lat, hr_rep rep, hr_prec prec, hr_op op, int n_rhs);

/* Full operator (Sec. 2.1): out = D in on all V sites; in/out are full packed
 * spinors (HR_FULL layout), gauge is packed with the same rep and prec. */
hr_status hr_dirac_apply(hr_ctx *ctx, hr_lattice lat, double m0, hr_rep rep, hr_prec prec,
                         const void *gauge, const void *in, void *out, hr_stream stream);

/* Even-odd operators (Sec. 2.1).  HR_OP_HOP: out (parity out_parity) =
 * -1/2 H in (in has the other parity); the SCHUR ops take and return even
 * vectors and need `work` of hr_dirac_workspace_bytes (odd temporaries).
 * n_rhs >= 1 vectors in the multi-RHS layout share each link load. */
hr_status hr_dirac_eo(hr_ctx *ctx, hr_lattice lat, double m0, hr_rep rep, hr_prec prec,
                      hr_parity out_parity, hr_op op, int n_rhs, const void *gauge, const void *in,
                      void *out, void *work, size_t work_bytes, hr_stream stream);

/* ---------------------------------------------------------------------- */
/* solvers                                                                 */
/* ---------------------------------------------------------------------- */

typedef struct {
    double tol;            /* stop when |b - A x| / |b| <= tol (true residual, FP64) */
    int maxiter;           /* cap on operator applications of A = Mhat^+ Mhat        */
    hr_prec inner_prec;    /* HR_F64: plain FP64 CG; HR_F32/HR_F16: mixed precision    */
    double reliable_delta; /* mixed precision: reliable update when |r| < delta max|r|  */
    int n_rhs;             /* independent right-hand sides solved together (>= 1)      */
    int x0_is_guess;       /* 1: x holds an initial guess; 0: start from x = 0          */
    int check_every;       /* 0: the device runs the whole loop (one graph launch, a  */
                           /* conditional WHILE node; reliable updates in IF nodes);   */
                           /* N > 0: replay a graph of N iterations, host check after */
                           /* each.  Either way at most maxiter iterations run.        */
} hr_solver_opts;

typedef struct {
    int iters;                 /* CG iterations (applications of A), max over RHS     */
    int n_reliable_updates;    /* FP64 residual recomputations                        */
    double true_rel_residual;  /* |b - A x| / |b| recomputed in FP64, max over RHS    */
    double seconds;            /* wall time of the solve on the stream                */
} hr_solve_info;

/* Default options: tol 1e-10, maxiter 20000, FP64, delta 0.1, 1 RHS. */
hr_solver_opts hr_solver_default_opts(void);

/* Work bytes for hr_cg_solve with these options. */
size_t hr_cg_workspace_bytes(hr_lattice lat, hr_rep rep, const hr_solver_opts *opts);

/* Solve Mhat^+ Mhat x = b on even sites by CG (Sec. 1 "inverters"; the
 * even-odd preconditioned operator of Sec. 2.1).  gauge: packed HR_F64 gauge
 * of `rep`; b, x: packed HR_F64 even spinors (n_rhs of them).  Low-precision
 * gauge copies for the mixed solver are made inside `work`.  Mixed precision
 * follows the reliable-update scheme: the inner recurrence runs in
 * inner_prec, and whenever |r| falls by reliable_delta the residual is
 * recomputed from the accumulated solution.  With HR_F16 inner, that
 * recomputation is FP32 (r_ref - A x_mid, x_mid the correction since the
 * last FP64 residual r_ref) until |r| has fallen by 1e-4 from r_ref, and FP64
 * (r = b - A x) then and at convergence; HR_F32 inner always recomputes in
 * FP64.  A right-hand side stops only on its FP64 residual, and
 * info->n_reliable_updates counts the FP64 recomputations.  Synchronises the
 * stream before returning (it reads the residuals); info may be NULL.
 * Every right-hand side is rescaled inside `work` by the power of two that
 * brings its largest component into [0.5, 1) (exact: the iterates are the
 * same numbers in other units), so the solve does not depend on the scale of
 * b; x is returned in the caller's units.  Returns HR_ERR_NOT_CONVERGED if
 * maxiter is reached (x = last iterate); HR_ERR_UNSUPPORTED if a right-hand
 * side's largest component is nonzero but below 2^-100 (its pairs have lost
 * low bits already) or a value packed since the last check exceeded 2^120,
 * HR_ERR_NUMERIC if one was NaN or Inf (hr_ctx_status). */
hr_status hr_cg_solve(hr_ctx *ctx, hr_lattice lat, double m0, hr_rep rep,
                      const hr_solver_opts *opts, const void *gauge, const void *b, void *x,
                      hr_solve_info *info, void *work, size_t work_bytes, hr_stream stream);

/* Full-lattice systems solved through the even-odd preconditioned operator. */
typedef enum { HR_SYSTEM_D = 0, HR_SYSTEM_DDAG_D = 1 } hr_system;

/* Work bytes for hr_solve_full (0 if the options are invalid; n_rhs must be 1). */
size_t hr_solve_full_workspace_bytes(hr_lattice lat, hr_rep rep, const hr_solver_opts *opts, hr_system system);

/* Solve D x = b (HR_SYSTEM_D) or D^+ D x = b (HR_SYSTEM_DDAG_D) on all sites
 * through the even-odd reduction of Sec. 2.1: the source bhat = b_e - D_eo b_o /
 * (4+m0), the Schur system Mhat x_e = bhat solved by hr_cg_solve on
 * Mhat^+ Mhat x_e = Mhat^+ bhat (opts: tol, maxiter, inner precision,
 * reliable_delta; n_rhs = 1), and the odd sites x_o = (b_o - D_oe x_e) /
 * (4+m0); D^+ D is two such solves, x = D^-1 g5 D^-1 g5 b.  gauge: packed
 * HR_F64 gauge of `rep`; b, x: full packed HR_F64 spinors (HR_FULL layout).
 * info->true_rel_residual = |b - op x| / |b| of the full system, recomputed in
 * FP64; iters and reliable updates are summed over the Schur solves.
 * Synchronises the stream.  Errors as hr_cg_solve (HR_ERR_NOT_CONVERGED if a
 * Schur solve misses tol within maxiter). */
hr_status hr_solve_full(hr_ctx *ctx, hr_lattice lat, double m0, hr_rep rep, const hr_solver_opts *opts,
                        hr_system system, const void *gauge, const void *b, void *x, hr_solve_info *info,
                        void *work, size_t work_bytes, hr_stream stream);

/* ---------------------------------------------------------------------- */
/* clover and exponential-clover site terms (Sec. 2.2)                      */
/* ---------------------------------------------------------------------- */

/* Sec. 2.2 adds the site-diagonal clover term (Sheikholeslami-Wohlert) or its
 * exponential form (Francis et al.) and precomputes it, with its inverse, once
 * per gauge field; it states no formula.  With Q_mn(x) the four plaquette
 * leaves of the (mu, nu) plane at x (mu-first), F_mn = (Q_mn - Q_mn^+)/8,
 * s_mn = (i/2)[g_mu, g_nu] and C = (i/4) sum_{mu != nu} s_mn F_mn:
 *   HR_CLOVER_SW:  A(x) = (4 + m0) + c_sw C(x)
 *   HR_CLOVER_EXP: A(x) = (4 + m0) exp(c_sw C(x) / (4 + m0))
 * and the operator is D = A - H/2, its Schur form on even sites
 * Mhat = A_ee - H_eo A_oo^-1 H_oe / 4, Mhat^+ = g5 Mhat g5.  m0 and c_sw are
 * baked into the packed field: the *_clover calls take no m0. */
typedef enum { HR_CLOVER_SW = 0, HR_CLOVER_EXP = 1 } hr_clover_kind;

/* Bytes of a packed clover field: A and A^-1 on both parities, two Hermitian
 * (2 nc) x (2 nc) blocks per site (chiral halves), HR_F64 (double-float pairs)
 * or HR_F32; 0 for HR_F16 or an invalid lattice.  The FP16 operators use the
 * HR_F32 field.  HR_ADJ and HR_ADJ_MAT share the adjoint layout. */
size_t hr_clover_packed_bytes(hr_lattice lat, hr_rep rep, hr_prec prec);

/* Build the packed clover field of `rep` from the canonical gauge (device,
 * double[4][V][4], the links as they are: boundary signs cancel around the
 * leaves) in FP64 arithmetic on the GPU.  HR_CLOVER_SW inverts each block by
 * Gauss-Jordan elimination (HR_ERR_NUMERIC if one is singular);
 * HR_CLOVER_EXP takes the exponential and its inverse exp(-...) by scaling
 * and squaring.  Synchronises the stream (it reads the singularity flag). */
hr_status hr_clover_build(hr_ctx *ctx, hr_lattice lat, hr_rep rep, hr_prec prec, hr_clover_kind kind,
                          double m0, double c_sw, const double *canonical, void *clover, hr_stream stream);

/* out = A in (inverse = 0) or A^-1 in (inverse != 0) on the sites of
 * `parity` (HR_EVEN / HR_ODD): packed spinors of precision prec with n_rhs
 * right-hand sides; clover: the packed field in the clover precision of prec
 * (HR_F64 for HR_F64, HR_F32 otherwise).  in may equal out. */
hr_status hr_clover_apply(hr_ctx *ctx, hr_lattice lat, hr_rep rep, hr_prec prec, hr_parity parity, int inverse,
                          int n_rhs, const void *clover, const void *in, void *out, hr_stream stream);

/* out = D in = A in - H in / 2 on all sites (HR_FULL packed spinors): two hop
 * launches with A applied to the local term in their epilogue. */
hr_status hr_dirac_apply_clover(hr_ctx *ctx, hr_lattice lat, hr_rep rep, hr_prec prec, const void *gauge,
                                const void *clover, const void *in, void *out, hr_stream stream);

/* hr_dirac_eo with the clover site term: HR_OP_SCHUR, HR_OP_SCHUR_DAG and
 * HR_OP_NORMAL apply Mhat = A_ee - H_eo A_oo^-1 H_oe / 4 (A_oo^-1 in the first
 * hop's epilogue, A_ee in the second's); HR_OP_HOP is the plain hop.  Work
 * bytes as hr_dirac_workspace_bytes. */
hr_status hr_dirac_eo_clover(hr_ctx *ctx, hr_lattice lat, hr_rep rep, hr_prec prec, hr_parity out_parity,
                             hr_op op, int n_rhs, const void *gauge, const void *clover, const void *in,
                             void *out, void *work, size_t work_bytes, hr_stream stream);

/* Work bytes of hr_cg_solve_clover (the mixed solvers keep an HR_F32 copy of
 * the clover field in it). */
size_t hr_cg_clover_workspace_bytes(hr_lattice lat, hr_rep rep, const hr_solver_opts *opts);

/* hr_cg_solve on Mhat^+ Mhat with the clover site term; clover: the packed
 * HR_F64 field (hr_clover_build).  Same options, errors and info. */
hr_status hr_cg_solve_clover(hr_ctx *ctx, hr_lattice lat, hr_rep rep, const hr_solver_opts *opts,
                             const void *gauge, const void *clover, const void *b, void *x, hr_solve_info *info,
                             void *work, size_t work_bytes, hr_stream stream);

/* Work bytes of hr_solve_full_clover. */
size_t hr_solve_full_clover_workspace_bytes(hr_lattice lat, hr_rep rep, const hr_solver_opts *opts,
                                            hr_system system);

/* hr_solve_full with the clover site term: bhat = b_e + H_eo A_oo^-1 b_o / 2,
 * Mhat x_e = bhat by hr_cg_solve_clover, x_o = A_oo^-1 (b_o + H_oe x_e / 2);
 * D^+ D = g5 D g5 D as for the Wilson operator.  clover: packed HR_F64 field. */
hr_status hr_solve_full_clover(hr_ctx *ctx, hr_lattice lat, hr_rep rep, const hr_solver_opts *opts,
                               hr_system system, const void *gauge, const void *clover, const void *b, void *x,
                               hr_solve_info *info, void *work, size_t work_bytes, hr_stream stream);

/* ---- the clover term in the HMC (fundamental links; SW and exponential forms) ----
 * The paper measures the clover operator (Sec. 2.2) and names the HMC as its
 * consumer; these calls give the molecular-dynamics force and action of the
 * term.  With the site term, two flavours weigh det(D^+ D) = det(A_oo)^2
 * det(Mhat^+ Mhat): S = S_pf + S_det, S_pf = Re<eta, (Mhat^+ Mhat)^-1 eta>,
 * S_det = -2 sum_{x odd} log det A(x).  Forces are dS/dw_a under
 * U_mu(x) -> exp(i w.s/2) U_mu(x), [4][V][3] doubles, accumulated (+=), as
 * hr_force.  The derivative of C(x) runs through the 8 leaves of each plane
 * that hold a link (one thread per link, native FP64). */

/* Work bytes of hr_clover_insertion_force and hr_clover_fermion_force. */
size_t hr_clover_force_workspace_bytes(hr_lattice lat);

/* force += coeff c_sw d/dw Re sum_x tr[C(x) lam(x)]: gauge is the canonical
 * FP64 field (double[4][V][4], without boundary signs, which cancel around
 * the leaves); lam is a device array of complex doubles [V][8][8] (row and
 * column index spin * 2 + colour, lexicographic sites). */
hr_status hr_clover_insertion_force(hr_ctx *ctx, hr_lattice lat, double c_sw, const double *gauge,
                                    const double *lam, double coeff, double *force, void *work, size_t work_bytes,
                                    hr_stream stream);

/* force += coeff dS/dw for S_pf (and S_det if with_det) at the links of
 * gauge (canonical) / gauge_packed (hr_gauge_pack of the same links, HR_FUND
 * HR_F64) and clover (HR_FUND HR_F64, hr_clover_build with kind, m0, c_sw of
 * those links), X = (Mhat^+ Mhat)^-1 eta (packed HR_F64 even): with
 * Y = Mhat X (or the given even Y, nullable: then the call differentiates
 * -2 Re<Y, Mhat X> at fixed X, Y, as the Hasenbusch ratio term needs),
 * Z = A_oo^-1 H_oe X, W = A_oo^-1 H_eo^+ Y, the hops give
 * 1/2 dRe<(Y, W), H (X, Z)> (hr_force) and the site term c_sw times the
 * insertion force of Lam = -2 X Y^+ on even sites, -1/2 Z W^+ - 2 A^-1 [det]
 * on odd sites.  HR_CLOVER_EXP (A = (4+m0) exp(c_sw C / (4+m0))): the site
 * term takes Lam' = int_0^1 exp((1-s) X) Lam exp(s X) ds, X = c_sw C / (4+m0),
 * per chiral block from the eigen-decomposition of A (Jacobi), and S_det is a
 * constant (tr C = 0): with_det adds nothing.  lat.bc and lat.theta apply to
 * the hops. */
hr_status hr_clover_fermion_force(hr_ctx *ctx, hr_lattice lat, hr_clover_kind kind, double m0, double c_sw,
                                  const double *gauge, const void *gauge_packed, const void *clover, const void *X,
                                  const void *Y, int with_det, double coeff, double *force, void *work,
                                  size_t work_bytes, hr_stream stream);

/* *logdet = sum over the sites of `parity` of log det A(x) (both chiral
 * blocks, by Cholesky) from an FP64 clover field (HR_FUND or HR_ADJ).
 * HR_ERR_NUMERIC if a block is not positive definite.  Synchronises the
 * stream. */
hr_status hr_clover_logdet(hr_ctx *ctx, hr_lattice lat, hr_rep rep, const void *clover, hr_parity parity,
                           double *logdet, hr_stream stream);

/* ---------------------------------------------------------------------- */
/* HMC molecular dynamics (Sec. 1 and 2.1 name the HMC as the consumer)      */
/* ---------------------------------------------------------------------- */

/* SU(2) with two flavours of even-odd preconditioned Wilson fermions in the
 * fundamental representation; the paper writes no formula, these are the
 * textbook ones:
 *   S_g = beta sum_{x, mu<nu} (1 - 1/2 Re tr P_mn(x))   (Wilson plaquette)
 *   S_f = Re <eta, (Mhat^+ Mhat)^-1 eta>               (pseudofermion on even sites)
 *   H = 1/2 sum p_a(x,mu)^2 + S_g + S_f, momenta p in su(2) (3 reals per link),
 *   flow U -> exp(i eps p.s/2) U, p -> p - eps F, F_a = dS/dw_a under
 *   U -> exp(i w.s/2) U (the force convention of hr_force).
 * Links: canonical quaternions, device double[4][V][4]; momenta and forces:
 * device double[4][V][3], lexicographic sites. */

/* force[mu][x][a] += coeff * dS_g/dw_a (F_a = beta/2 vec(U V)_a, V the staple sum). */
hr_status hr_gauge_force(hr_ctx *ctx, hr_lattice lat, double beta, const double *gauge, double coeff,
                         double *force, hr_stream stream);
/* *action = S_g (synchronises the stream). */
hr_status hr_gauge_action(hr_ctx *ctx, hr_lattice lat, double beta, const double *gauge, double *action,
                          hr_stream stream);
/* U_mu(x) <- exp(i eps p_mu(x).s/2) U_mu(x) for every link, renormalised to unit length. */
hr_status hr_link_update(hr_ctx *ctx, hr_lattice lat, double eps, const double *mom, double *gauge,
                         hr_stream stream);
/* mom <- mom - eps force. */
hr_status hr_mom_update(hr_ctx *ctx, hr_lattice lat, double eps, const double *force, double *mom,
                        hr_stream stream);
/* *energy = 1/2 sum mom^2 (synchronises the stream). */
hr_status hr_kinetic_energy(hr_ctx *ctx, hr_lattice lat, const double *mom, double *energy, hr_stream stream);

typedef enum { HR_INTEGRATOR_LEAPFROG = 0, HR_INTEGRATOR_OMELYAN = 1 } hr_integrator;

typedef struct {
    double beta;              /* gauge coupling                                       */
    double m0;                /* Wilson mass of the two fundamental flavours           */
    int fermions;             /* 0: pure gauge; 1: with the pseudofermion eta          */
    int n_steps;              /* integration steps per trajectory (>= 1)               */
    double tau;               /* trajectory length (> 0)                               */
    hr_integrator integrator; /* leapfrog, or Omelyan's minimum-norm 2nd-order scheme  */
    hr_solver_opts solver;    /* CG of the force and of S_f (tol, inner precision, ...) */
    int hasenbusch;           /* 1: Hasenbusch mass preconditioning (two pseudofermions) */
    double m0_hasenbusch;     /* its heavier mass                                      */
    int n_steps_gauge;        /* two time scales: gauge-force steps per link update of */
                              /* the fermion integrator (> 1); 0 or 1: one time scale  */
    int clover;               /* 1: clover fermions, c_sw and clover_kind below        */
    double c_sw;              /* their coefficient                                     */
    hr_clover_kind clover_kind; /* HR_CLOVER_SW (0) or HR_CLOVER_EXP                   */
} hr_hmc_params;

typedef struct {
    double dH;                                         /* H(end) - H(start)          */
    double kinetic_start, kinetic_end;
    double gauge_action_start, gauge_action_end;
    double fermion_action_start, fermion_action_end;
    double plaquette;                                  /* <1/2 tr P> at the end      */
    int cg_iters;                                      /* summed over the solves     */
    int solves;
    double seconds;                                    /* host wall time             */
} hr_hmc_info;

/* Work bytes of hr_hmc_trajectory (0 if the parameters are invalid). */
size_t hr_hmc_workspace_bytes(hr_lattice lat, const hr_hmc_params *prm);

/* One molecular-dynamics trajectory of n_steps steps of length tau / n_steps
 * from (gauge, mom), both updated in place; eta: packed HR_F64 even spinor
 * (prm->fermions; the caller draws it as Mhat^+ xi with P(xi) ~ exp(-xi^+ xi)),
 * NULL for pure gauge.  With prm->hasenbusch (Hasenbusch's mass
 * preconditioning, a standard HMC acceleration the paper cites in Sec. 2.2),
 * S_f = Re<eta, (Mhat_H^+ Mhat_H)^-1 eta> + Re<eta2, (Mhat^+ Mhat)^-1 eta2>,
 * eta2 = Mhat_H^+ phi, Mhat_H the Schur operator at m0_hasenbusch: eta is
 * drawn as Mhat_H^+ xi1 and phi (packed HR_F64 even) as
 * Mhat_H (Mhat_H^+ Mhat_H)^-1 Mhat^+ xi2; each force then takes two solves.  Leapfrog: p -= eps/2 F, U <- exp(i eps p) U,
 * p -= eps/2 F; Omelyan: p -= l eps F, U <- exp(i eps/2 p) U, p -= (1-2l) eps F,
 * U <- exp(i eps/2 p) U, p -= l eps F, l = 0.1931833275037836; the force of
 * the current links is reused between steps.  With n_steps_gauge = m > 1 and
 * fermions (Sexton and Weingarten's multiple time scales; the paper gives no
 * integrator), the kicks of that scheme use the pseudofermion force alone and
 * each of its link updates, of length t, becomes m steps of length t / m of
 * the same integrator driven by the gauge force alone: as many solves as
 * with m = 1, m times (leapfrog; 2m, Omelyan) as many gauge-force steps.
 * With prm->clover the fermions carry the site term of prm->clover_kind (Mhat = A_ee -
 * H_eo A_oo^-1 H_oe / 4, eta drawn as Mhat^+ xi with that Mhat): the clover
 * field is rebuilt from the links before each solve, S_f = Re<eta, (Mhat^+
 * Mhat)^-1 eta> - 2 sum_{odd} log det A, and the force is
 * hr_clover_fermion_force (hops, site term and det A_oo).
 * Each fermion force and S_f takes
 * one hr_cg_solve (from x = 0) on the packed links (lat.bc applies).  The
 * Metropolis test on info->dH and the draw of mom and eta are the caller's.
 * Synchronises the stream. */
hr_status hr_hmc_trajectory(hr_ctx *ctx, hr_lattice lat, const hr_hmc_params *prm, double *gauge, double *mom,
                            const void *eta, const void *phi, hr_hmc_info *info, void *work, size_t work_bytes,
                            hr_stream stream);

/* Work bytes of hr_cg_solve_batch for these lattices (0 if invalid). */
size_t hr_cg_batch_workspace_bytes(int n_lat, const hr_lattice *lats, hr_rep rep);

/* Solve Mhat^+ Mhat x_l = b_l for n_lat (1..64) independent lattices of any
 * sizes at once (FP64 CG, one RHS each, HR_FUND or HR_ADJ).  The paper notes
 * that SU(2) lattices below 16^4 lose efficiency to fixed overheads (Sec. 3);
 * here every CG phase is one persistent launch over a work list of all the
 * lattices' 128-site tiles, with per-lattice scalars and convergence flags on
 * the device; the iteration loop runs on the device as one CUDA graph
 * (check_every > 0: a graph of that many iterations with a host check after
 * each), and converged lattices drop out of the work.  gauges[l]:
 * packed HR_F64 gauge of lats[l]; b[l], x[l]: packed HR_F64 even spinors.
 * infos[l] (may be NULL) receives each lattice's iterations and true residual
 * (seconds = the whole batch).  Synchronises the stream.  Returns
 * HR_ERR_NOT_CONVERGED if any lattice misses tol within maxiter. */
hr_status hr_cg_solve_batch(hr_ctx *ctx, int n_lat, const hr_lattice *lats, double m0, hr_rep rep,
                            const hr_solver_opts *opts, const void *const *gauges, const void *const *b,
                            void *const *x, hr_solve_info *infos, void *work, size_t work_bytes,
                            hr_stream stream);

/* ---------------------------------------------------------------------- */
/* link derivatives                                                         */
/* ---------------------------------------------------------------------- */

/* The even-odd preconditioned operator is "used mainly in the HMC" (Sec. 2.1),
 * whose molecular dynamics needs the derivative of fermion bilinears with
 * respect to the links.  The paper writes no formula; these are the textbook
 * ones for the operator above.  Variation: U_mu(x) -> exp(i w.s/2) U_mu(x),
 * F_a = d/dw_a (the su(2) force), or the four quaternion components q_k of
 * U = sum_k q_k E_k (E_0 = 1, E_k = i s_k).  Outputs are accumulated (+=):
 * force double[4][V][3], grad double[4][V][4] (device, lexicographic sites).
 * Fundamental links only (HR_ERR_UNSUPPORTED otherwise); lat.bc and lat.theta
 * apply as in the operators. */

/* Work bytes of hr_fermion_force / hr_fermion_link_grad (five packed FP64
 * spinor halves); 0 for an invalid lattice. */
size_t hr_fermion_force_workspace_bytes(hr_lattice lat);

/* force += coeff * d/dw Re<L, Mhat^+ Mhat X> at fixed even fields X and L
 * (packed HR_F64 even spinors; L = NULL means L = X), gauge: packed HR_F64
 * fundamental links, m0 the Wilson mass of Mhat.  For the pseudofermion
 * action S = Re<eta, (Mhat^+ Mhat)^-1 eta> with X = (Mhat^+ Mhat)^-1 eta (the
 * solution of hr_cg_solve), dS/dw = -d/dw Re<X, Mhat^+ Mhat X>: call with
 * L = NULL, coeff = -1.  Internally, with c = 1/(4(4+m0)) and
 * H_eo^+ = g5 H_oe g5, Re<Y, dMhat Z> = -c dRe<(Y, H_eo^+ Y), H (Z, H_oe Z)>:
 * the call forms Mhat X (and Mhat L), the odd halves by hops, and applies
 * the hop derivative of hr_force once (L = X) or twice.  Asynchronous;
 * work: hr_fermion_force_workspace_bytes, 16-byte aligned. */
hr_status hr_fermion_force(hr_ctx *ctx, hr_lattice lat, double m0, hr_rep rep, const void *gauge, const void *X,
                           const void *L, double coeff, double *force, void *work, size_t work_bytes,
                           hr_stream stream);

/* As hr_fermion_force, with the derivative taken with respect to the
 * quaternion components: grad += coeff * d/dq Re<L, Mhat^+ Mhat X>.  The
 * gradient of x = (Mhat^+ Mhat)^-1 eta against a cotangent g is
 * -d/dq Re<lambda, Mhat^+ Mhat x> with lambda = (Mhat^+ Mhat)^-1 g: X = x,
 * L = lambda, coeff = -1. */
hr_status hr_fermion_link_grad(hr_ctx *ctx, hr_lattice lat, double m0, hr_rep rep, const void *gauge,
                               const void *X, const void *L, double coeff, double *grad, void *work,
                               size_t work_bytes, hr_stream stream);

/* The hop derivative itself (the building block of the calls above; Sec. 2.1
 * defines the hopping term H whose links it varies):
 * force[mu][x][a] += beta * d Re<a_f, H b_f> / d w_a.  The two terms of H that
 * hold U_mu(x) are a(x)^+ (1-g_mu) U b(x+mu) and a(x+mu)^+ (1+g_mu) U^+ b(x);
 * with M1 = sum_s b(x+mu)_s [((1-g_mu) a(x))_s]^+ and
 * M2 = sum_s b(x)_s [((1+g_mu) a(x+mu))_s]^+, F_a = Re tr[(i s_a/2)(U M1 - M2 U^+)].
 * a_f, b_f: full packed FP64 fundamental spinors; gauge: packed HR_F64
 * fundamental links (the boundary signs ride on them). */
hr_status hr_force(hr_ctx *ctx, hr_lattice lat, const void *gauge, const void *a_full,
                   const void *b_full, double beta, double *force, hr_stream stream);

/* The hop derivative with respect to the quaternion components (same terms as
 * hr_force): grad[mu][x][k] += beta * (Re tr[E_k M1] + Re tr[E_k^+ M2]), with
 * the boundary sign of lat.bc on the links of the last slice of each
 * antiperiodic direction (the call takes no gauge field: H is linear in U). */
hr_status hr_link_grad(hr_ctx *ctx, hr_lattice lat, const void *a_full, const void *b_full,
                       double beta, double *grad, hr_stream stream);

/* ---------------------------------------------------------------------- */
/* autotuning of the hop kernel's launch shape                              */
/* ---------------------------------------------------------------------- */

typedef struct {
    int variant;       /* 0: unrolled directions, operands in registers; 1: unrolled, cp.async
                          staged in shared memory; 2: generic looped directions, registers;
                          3: generic looped, staged; 4: loop over mu with switched projections,
                          registers; 5: switched, staged; 6: unrolled with the next direction's
                          operands prefetched into registers; 7: as 0, capped at 96
                          registers per thread (more resident warps); 8: tiled, the
                          near-direction neighbours bulk-copied (TMA) into shared memory;
                          9: as 8, 96 registers; 10: packed f32x2 FMAs, two numbers per
                          instruction (fundamental: the two colours; adjoint FP64: re and
                          im); 11: as 10, operands staged by cp.async one direction ahead
                          (fundamental, adjoint FP64 with quaternion links); 12, 13: 10,
                          11 for fundamental FP64 capped at 96 registers (12 for adjoint
                          FP64: 10 with up to 168 registers); 14: fundamental
                          binary16 with the spin projection in half2 arithmetic (only the
                          projected half spinor is widened to FP32, the neighbour's scale
                          rides on the accumulating FMAs); 15: as 14, 64 registers; 16:
                          fundamental FP32 / binary16 with two sites per thread, one in
                          each lane of the packed f32x2 FMAs; 17: as 16, 96 registers;
                          18, 19: 14, 15 with the next direction's operands staged by
                          cp.async in shared memory; 20, 21: fundamental FP32 /
                          binary16 with n_rhs >= 2 / 4, a chunk of 2 / 4 right-hand
                          sides per thread sharing the site's neighbour indices and
                          links; 22, 23: 14 with the next one / two directions'
                          operands loaded into registers ahead (80 / 96 registers).
                          The FP64 results of 8-13 are bit-identical to those
                          of 0. */
    int block;         /* threads per block                                               */
    double best_ms;    /* time of one hop launch with the chosen shape (median of 4)      */
    double default_ms; /* the same for the shape in use before tuning                     */
    int candidates;    /* shapes timed, both sweeps                                       */
} hr_tune_result;

/* Time every kernel variant and block size for the hop of this configuration
 * (rep, prec, extents, n_rhs) on the caller's buffers -- `out` (parity
 * out_parity) is overwritten with D_{p,1-p} in, `reps` timed launches per
 * shape; the four fastest are timed three more times, interleaved, and the
 * best median wins -- and use it for all later hop launches of the
 * configuration on this context (operators and solvers included).  A second
 * sweep, starting from that winner, times the reducing form the solvers
 * launch (the epilogue also reads an aux vector and reduces |out|^2 over the
 * grid; `out` serves as its aux) and keeps its own winner for those launches;
 * *result reports the plain hop's choice.  If the environment variable
 * HR_AUTOTUNE_CACHE names a file, both choices are written there as JSON (the
 * reducing one under the key suffixed ":fin") and read back by later
 * contexts; a plain key without its ":fin" entry serves both forms.
 * Synchronises the stream.
 * A lattice with twisted boundaries (hr_lattice.theta) runs one kernel
 * whatever the shape: the call returns HR_OK at once, *result zeroed.
 * (The paper measures a hand-tuned kernel, Sec. 3; tuning per shape is this
 * library's way to reach the bandwidth bound on each lattice.) */
hr_status hr_autotune_hop(hr_ctx *ctx, hr_lattice lat, hr_rep rep, hr_prec prec, hr_parity out_parity,
                          int n_rhs, const void *gauge, const void *in, void *out, int reps,
                          hr_tune_result *result, hr_stream stream);
/* The launch shape the context uses now for this configuration. */
hr_status hr_tune_lookup(hr_ctx *ctx, hr_lattice lat, hr_rep rep, hr_prec prec, int n_rhs, int *variant,
                         int *block);

/* ---------------------------------------------------------------------- */
/* vector utilities on packed FP64 spinors (n vectors of one parity)        */
/* ---------------------------------------------------------------------- */

/* *result (host) = sum |v|^2 over the packed even/odd FP64 field (n_rhs = 1).
 * Synchronises the stream. */
hr_status hr_norm2(hr_ctx *ctx, hr_lattice lat, hr_rep rep, const void *v, double *result,
                   hr_stream stream);
/* *re + i *im (host) = <a, b> = sum conj(a) b over the packed FP64 fields of
 * one parity (n_rhs = 1), accumulated in binary64 and summed in a fixed order
 * (deterministic).  Synchronises the stream. */
hr_status hr_dot(hr_ctx *ctx, hr_lattice lat, hr_rep rep, const void *a, const void *b, double *re, double *im,
                 hr_stream stream);
/* y = a*x + y on packed FP64 fields of one parity. */
hr_status hr_axpy(hr_ctx *ctx, hr_lattice lat, hr_rep rep, double a, const void *x, void *y,
                  hr_stream stream);
/* v = g5 v on a packed FP64 field of one parity (in place). */
hr_status hr_gamma5(hr_ctx *ctx, hr_lattice lat, hr_rep rep, void *v, hr_stream stream);

/* ---------------------------------------------------------------------- */
/* domain decomposition along time (Sec. 2.1.1)                            */
/* ---------------------------------------------------------------------- */

/* The paper distributes the lattice over GPUs: each computes its inner sites
 * while the boundary data travels, then its boundary sites (Sec. 2.1.1; the
 * weak and strong scaling of Table 1).  Here the lattice (T, L1, L2, L3) is
 * split along time into n slabs of T_loc = T / n slices (T_loc even), one per
 * rank, each an ordinary local lattice (T_loc, L1, L2, L3) packed and hopped
 * with the calls above.  A local hop (hr_dirac_eo, HR_OP_HOP) wraps time
 * inside the slab; every term is right except the time hops of the two face
 * slices.  Per hop, each rank
 *   1. packs its faces of the input field (hr_dd_pack_faces),
 *   2. sends to_lower to the rank below (it arrives there as from_upper) and
 *      to_upper to the rank above (arriving as from_lower), periodic in the
 *      rank index -- a device copy when two slabs share a GPU, NCCL send /
 *      receive into the receiver's own buffer across GPUs,
 *   3. runs the local hop meanwhile (the inner sites need nothing remote),
 *   4. after the exchange, replaces the wrapped time terms of its face sites
 *      by the received ones (hr_dd_hop_boundary).
 * Boundary conditions: pack the local gauge field with lat.bc bit 0 only on
 * the last slab (it holds the global time boundary) and the spatial bits on
 * every slab; a twist in time is not supported (HR_ERR_UNSUPPORTED).  One
 * right-hand side.  Face layout: 4 NC reals per face site (the two spins of
 * a projected half spinor), V3/2 face sites (V3 = L1 L2 L3) numbered by their
 * even-odd index within the slice; FP64 faces hold (hi, lo) float pairs. */

/* Bytes of one face buffer for the local lattice `local` (0 if invalid). */
size_t hr_dd_face_bytes(hr_lattice local, hr_rep rep, hr_prec prec);

/* The two faces of the packed input field `in` (sites of in_parity of the
 * local lattice): to_lower = P-_0 psi on the slice t = 0 and to_upper =
 * U_0(x)^+ P+_0 psi(x) on t = T_loc - 1, with P-+_0 the projections of
 * (1 -+ g_0).  gauge: the packed local gauge field of rep and prec. */
hr_status hr_dd_pack_faces(hr_ctx *ctx, hr_lattice local, hr_rep rep, hr_prec prec, hr_parity in_parity,
                           const void *gauge, const void *in, void *to_lower, void *to_upper, hr_stream stream);

/* After out = -1/2 H_{p,1-p} in on the local lattice (hr_dirac_eo with
 * HR_OP_HOP, out_parity p), give the face sites of out their time hops from
 * the neighbouring slabs: out += -1/2 (1 - g_0) U_0(x) [from_upper - P-_0 psi
 * (wrapped)] on t = T_loc - 1 and out += -1/2 (1 + g_0) [from_lower - U_0^+
 * P+_0 psi (wrapped)] on t = 0.  from_upper / from_lower: the faces the rank
 * above / below packed (its to_lower / to_upper) from its own input field. */
hr_status hr_dd_hop_boundary(hr_ctx *ctx, hr_lattice local, hr_rep rep, hr_prec prec, hr_parity out_parity,
                             const void *gauge, const void *in, const void *from_lower, const void *from_upper,
                             void *out, hr_stream stream);

/* ---------------------------------------------------------------------- */
/* calibration (a measurement service for benchmarks; no paper counterpart) */
/* ---------------------------------------------------------------------- */

/* The FP32 FMA pipe's delivered rate on the context's device, in lane
 * operations per second (an FFMA counts 1, a packed f32x2 FMA 2): independent
 * FMA chains with shared multiplier and addend (the operand-reuse best case),
 * scalar into *scalar_lane_ops and packed into *paired_lane_ops, best of three
 * timed launches of about half a millisecond.  The FP64-class kernels compute
 * with pairs of floats on this pipe, so their ALU roofline is this rate.
 * Synchronises the stream; uses the context's scratch. */
hr_status hr_fp32_fma_rate(hr_ctx *ctx, double *scalar_lane_ops, double *paired_lane_ops, hr_stream stream);

/* ---------------------------------------------------------------------- */
/* allocation-free reduction (a library service; the paper has no           */
/* counterpart)                                                             */
/* ---------------------------------------------------------------------- */

/* result[r] = |v_r|^2 for the n_rhs packed FP64 spinor fields of one parity
 * in v (multi-RHS layout when n_rhs > 1), written to the DEVICE array
 * `result` (n_rhs doubles) asynchronously on `stream`.
 *
 * For callers that may not allocate device memory at all -- hr_ctx_create
 * calls cudaMalloc, so they cannot hold a context -- this call needs neither
 * a context nor a workspace and calls no allocating routine.  Its scratch (the
 * block partial sums and a completion counter) is a fixed 256 KiB device
 * array inside the library, which every GPU that loads the library keeps
 * until the process exits; it has room for up to 32 right-hand sides.
 * The first call on a device sets the array up: it looks up the array's
 * device address, and under CUDA's default lazy module loading that is also
 * when the driver loads this part of the library and places the array in
 * device memory.  So make the first call before any stream capture and
 * before the process reserves the rest of the device memory for itself (or
 * run with CUDA_MODULE_LOADING=EAGER, which places it when the library is
 * loaded); later calls take no device memory.  The kernel runs on the
 * current device with that device's array: a stream of another device is
 * refused.  All calls share the array: calls that overlap on the GPU
 * (different streams or threads) race and return wrong sums, so serialise
 * them.  After a cudaDeviceReset the next call looks the address up again
 * only once a launch has failed: reload the library instead.  Errors (no
 * message is recorded, there is no context): n_rhs > 32 -> HR_ERR_WORKSPACE;
 * n_rhs not a power of two, odd or oversized extents -> HR_ERR_UNSUPPORTED;
 * extent < 2, bc outside [0, 15], a non-finite theta, bad rep, null or
 * misaligned pointer, a stream of another device -> HR_ERR_INVALID_ARG; a
 * failed launch -> HR_ERR_CUDA. */
hr_status hr_norm2_noalloc(hr_lattice lat, hr_rep rep, int n_rhs, const void *v, double *result,
                           hr_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* HIREP_GB300_H */
