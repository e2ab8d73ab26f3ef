// hr_batch.cu -- CG on Mhat^+ Mhat for many lattices of different sizes at once.
//
// The paper advises against SU(2) local lattices below 16^4 because fixed
// overheads dominate there (Sec. 3); on one GB300 a small lattice leaves most
// of the 152 SMs idle and a solve is bound by launch latency.  This solver runs
// every lattice of a batch inside the same launches: each CG phase (the four
// hops of Mhat^+ Mhat, the x/r update, the p update) is one persistent launch
// whose blocks walk a work list of (lattice, 128-site tile) entries.  Each
// lattice keeps its own device scalars (alpha, beta, |r|^2, convergence flag);
// reductions finish per lattice in its last tile (deterministic tile order);
// converged lattices drop out of the work.  The iteration loop runs on the
// device as one CUDA graph: a conditional WHILE node over passes of 8
// iterations, its condition set from the lattices' done flags.
#include <cmath>
#include <cstring>
#include <vector>

#include "hr_hop_x2.cuh"

using namespace hr;

namespace {

constexpr int kTile = 128; // sites per tile = threads per block
constexpr int kMaxLattices = 64;
constexpr int kBatchCounters = 4;

struct BatchLat {
    Geom g;
    const void *gauge;
    const void *b;
    void *x, *r, *p, *q, *u, *t;
    double *scal;       // S_NSLOTS x kMaxRhsSlots doubles
    double *partials;   // one per tile
    unsigned *counters; // kBatchCounters
    int tile0, ntiles;
    coef2 A, negc;      // 4 + m0 and -1/(4(4+m0))
};

struct BatchArgs {
    const BatchLat *lat;
    int nlat;
    int total_tiles;
    int use_x;       // hop phases act on x instead of p (true residual)
    int ignore_done; // run converged lattices too (true residual)
    float unit, nil; // 1 and 0 at run time (the paired arithmetic's multipliers)
};

__device__ __forceinline__ int find_lat(const BatchLat *L, int n, int tile)
{
    int l = 0;
    while (l + 1 < n && tile >= L[l + 1].tile0) ++l;
    return l;
}

// Block sum of v; the last tile of the lattice adds the tile partials in order
// and runs the scalar update `fin` (and `fin2` after it, if nonzero).
__device__ void tile_reduce(double v, const BatchLat &L, int tile, int counter, int fin, int fin2)
{
    __shared__ double wsum[kTile]; // >= 32 per warp for sum_partials
    __shared__ bool last;
    __shared__ double sums[32];
    v = warp_sum_strided(v, 1);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int w = 0; w < kTile / 32; ++w) s += wsum[w];
        L.partials[tile - L.tile0] = s;
        __threadfence();
        unsigned prev = atomicAdd(L.counters + counter, 1u);
        last = (prev == (unsigned)L.ntiles - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    sum_partials(L.partials, (unsigned)L.ntiles, 1, sums, wsum);
    if (threadIdx.x == 0) L.counters[counter] = 0u;
    finish_reduction(fin, sums, 1, L.scal);
    if (fin2) {
        __syncthreads();
        finish_reduction(fin2, sums, 1, L.scal);
    }
    __syncthreads();
}

// PHASE 0: t = H_oe v            1: u = A v - c H_eo t, |u|^2 -> alpha
//       2: t = H_oe g5 u         3: q = A u - c g5 H_eo t        (v = p, or x)
template <int REP, int PHASE>
__global__ void __launch_bounds__(kTile) k_batch_hop(BatchArgs B)
{
    using T = dd;
    for (int tile = blockIdx.x; tile < B.total_tiles; tile += gridDim.x) {
        const int l = find_lat(B.lat, B.nlat, tile);
        const BatchLat &L = B.lat[l];
        if (!B.ignore_done && sc(L.scal, S_FLAGS, F_DONE) != 0.0) continue;
        const void *v = B.use_x ? (const void *)L.x : (const void *)L.p;
        HopArgs a{};
        a.g = L.g;
        a.gauge = L.gauge;
        a.red = RedSlot{nullptr, nullptr};
        a.scal = L.scal;
        a.fin = (PHASE == 1) ? kFinAlpha : kFinNone;
        coef2 zero = {0.f, 0.f}, one = {1.f, 0.f};
        if (PHASE == 0) { a.p = 1; a.in = v; a.out = L.t; a.alpha = zero; a.beta = one; a.beta_pow2 = 1; }
        if (PHASE == 1) { a.p = 0; a.in = L.t; a.aux = v; a.out = L.u; a.alpha = L.A; a.beta = L.negc; }
        if (PHASE == 2) { a.p = 1; a.in = L.u; a.out = L.t; a.alpha = zero; a.beta = one; a.beta_pow2 = 1; a.g5_in = 1; }
        if (PHASE == 3) { a.p = 0; a.in = L.t; a.aux = L.u; a.out = L.q; a.alpha = L.A; a.beta = L.negc; a.g5_out = 1; }
        const T be = Real<T>::from_coef(a.beta);
        const T bu = a.g5_out ? -be : be;
        const T al = Real<T>::from_coef(a.alpha);
        SqAcc<T> red;
        const int j = (tile - L.tile0) * kTile + threadIdx.x;
        if (j < L.g.vh) {
            if constexpr (REP == kRepFund) {
                // the paired (f32x2) double-float arithmetic of the single-lattice
                // hop: the same sums in the same order, half the instructions
                constexpr bool NEG = PHASE == 2;
                const K2 k = make_k2(B.unit, B.nil);
                SiteNb nb;
                site_neighbours(a.g, j, a.p, nb);
                cdd2 acc[4];
                x2_dir<0, true, NEG>(a, k, j, 0, nb, acc);
                x2_dir<1, false, NEG>(a, k, j, 0, nb, acc);
                x2_dir<2, false, NEG>(a, k, j, 0, nb, acc);
                x2_dir<3, false, NEG>(a, k, j, 0, nb, acc);
                x2_epilogue(a, j, acc, al, be, bu, red);
            } else {
                hop_site<REP, kF64>(a, j, al, be, bu, red);
            }
        }
        if (PHASE == 1) tile_reduce(red.get(), L, tile, 0, kFinAlpha, 0);
    }
}

template <int NC>
__global__ void __launch_bounds__(kTile) k_batch_xr(BatchArgs B)
{
    using T = dd;
    for (int tile = blockIdx.x; tile < B.total_tiles; tile += gridDim.x) {
        const int l = find_lat(B.lat, B.nlat, tile);
        const BatchLat &L = B.lat[l];
        if (sc(L.scal, S_FLAGS, F_DONE) != 0.0) continue;
        const T al = Real<T>::from_double(sc(L.scal, S_ALPHA, 0));
        SqAcc<T> red;
        const int j = (tile - L.tile0) * kTile + threadIdx.x;
        if (j < L.g.vh) {
            cpx<T> xv[4][NC], pv[4][NC], rv[4][NC], qv[4][NC];
            load_spinor<NC, kF64>(L.x, L.g.nblk_s, j, xv);
            load_spinor<NC, kF64>(L.p, L.g.nblk_s, j, pv);
            load_spinor<NC, kF64>(L.r, L.g.nblk_s, j, rv);
            load_spinor<NC, kF64>(L.q, L.g.nblk_s, j, qv);
#pragma unroll
            for (int s = 0; s < 4; ++s)
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    xv[s][c].re += al * pv[s][c].re;
                    xv[s][c].im += al * pv[s][c].im;
                    rv[s][c].re -= al * qv[s][c].re;
                    rv[s][c].im -= al * qv[s][c].im;
                    red.add(rv[s][c].re);
                    red.add(rv[s][c].im);
                }
            store_spinor<NC, kF64>(L.x, L.g.nblk_s, j, xv);
            store_spinor<NC, kF64>(L.r, L.g.nblk_s, j, rv);
        }
        tile_reduce(red.get(), L, tile, 1, kFinBeta, 0);
    }
}

template <int NC>
__global__ void __launch_bounds__(kTile) k_batch_p(BatchArgs B)
{
    using T = dd;
    for (int tile = blockIdx.x; tile < B.total_tiles; tile += gridDim.x) {
        const int l = find_lat(B.lat, B.nlat, tile);
        const BatchLat &L = B.lat[l];
        if (sc(L.scal, S_FLAGS, F_DONE) != 0.0) continue;
        const T be = Real<T>::from_double(sc(L.scal, S_BETA, 0));
        const int j = (tile - L.tile0) * kTile + threadIdx.x;
        if (j < L.g.vh) {
            cpx<T> pv[4][NC], rv[4][NC];
            load_spinor<NC, kF64>(L.p, L.g.nblk_s, j, pv);
            load_spinor<NC, kF64>(L.r, L.g.nblk_s, j, rv);
#pragma unroll
            for (int s = 0; s < 4; ++s)
#pragma unroll
                for (int c = 0; c < NC; ++c)
                    pv[s][c] = {rv[s][c].re + be * pv[s][c].re, rv[s][c].im + be * pv[s][c].im};
            store_spinor<NC, kF64>(L.p, L.g.nblk_s, j, pv);
        }
    }
}

// x = 0, r = p = b, |b|^2 -> bb, stop, and the initial |r|^2
template <int NC>
__global__ void __launch_bounds__(kTile) k_batch_start(BatchArgs B)
{
    using T = dd;
    for (int tile = blockIdx.x; tile < B.total_tiles; tile += gridDim.x) {
        const int l = find_lat(B.lat, B.nlat, tile);
        const BatchLat &L = B.lat[l];
        SqAcc<T> red;
        const int j = (tile - L.tile0) * kTile + threadIdx.x;
        if (j < L.g.vh) {
            cpx<T> bv[4][NC], z[4][NC];
            load_spinor<NC, kF64>(L.b, L.g.nblk_s, j, bv);
#pragma unroll
            for (int s = 0; s < 4; ++s)
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    z[s][c] = {T(0.f), T(0.f)};
                    red.add(bv[s][c].re);
                    red.add(bv[s][c].im);
                }
            store_spinor<NC, kF64>(L.x, L.g.nblk_s, j, z);
            store_spinor<NC, kF64>(L.r, L.g.nblk_s, j, bv);
            store_spinor<NC, kF64>(L.p, L.g.nblk_s, j, bv);
        }
        tile_reduce(red.get(), L, tile, 2, kFinBB, kFinInit);
    }
}

// r = b - q (q = A x), |r|^2 -> S_OUT
template <int NC>
__global__ void __launch_bounds__(kTile) k_batch_residual(BatchArgs B)
{
    using T = dd;
    for (int tile = blockIdx.x; tile < B.total_tiles; tile += gridDim.x) {
        const int l = find_lat(B.lat, B.nlat, tile);
        const BatchLat &L = B.lat[l];
        SqAcc<T> red;
        const int j = (tile - L.tile0) * kTile + threadIdx.x;
        if (j < L.g.vh) {
            cpx<T> bv[4][NC], qv[4][NC];
            load_spinor<NC, kF64>(L.b, L.g.nblk_s, j, bv);
            load_spinor<NC, kF64>(L.q, L.g.nblk_s, j, qv);
#pragma unroll
            for (int s = 0; s < 4; ++s)
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    cpx<T> d = csub(bv[s][c], qv[s][c]);
                    red.add(d.re);
                    red.add(d.im);
                }
        }
        tile_reduce(red.get(), L, tile, 3, kFinStore, 0);
    }
}

struct GraphExec {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t e = nullptr;
    ~GraphExec()
    {
        if (e) cudaGraphExecDestroy(e);
        if (g) cudaGraphDestroy(g);
    }
};

struct BatchPlan {
    size_t bytes = 0;
    std::vector<size_t> vec_off, scal_off, part_off, cnt_off;
    size_t desc_off = 0;
    std::vector<Geom> geoms;
    int total_tiles = 0;
};

BatchPlan plan_batch(int n, const hr_lattice *lats, int rep)
{
    BatchPlan P;
    size_t off = 0;
    auto take = [&](size_t b) {
        size_t o = off;
        off += (b + 255) & ~(size_t)255;
        return o;
    };
    P.desc_off = take(sizeof(BatchLat) * (size_t)n);
    for (int l = 0; l < n; ++l) {
        Geom g = make_geom(lats[l], 1);
        P.geoms.push_back(g);
        size_t h = spinor_half_bytes(g, rep, kF64);
        P.vec_off.push_back(take(6 * h)); // r p q u t (+ spare)
        P.scal_off.push_back(take(sizeof(double) * S_NSLOTS * kMaxRhsSlots));
        int nt = (g.vh + kTile - 1) / kTile;
        P.part_off.push_back(take(sizeof(double) * nt));
        P.cnt_off.push_back(take(sizeof(unsigned) * kBatchCounters));
        P.total_tiles += nt;
    }
    P.bytes = off;
    return P;
}

template <int REP>
hr_status batch_launch_iteration(hr_ctx *ctx, const BatchArgs &B, int grid, cudaStream_t s)
{
    constexpr int NC = RepTraits<REP>::NC;
    k_batch_hop<REP, 0><<<grid, kTile, 0, s>>>(B);
    k_batch_hop<REP, 1><<<grid, kTile, 0, s>>>(B);
    k_batch_hop<REP, 2><<<grid, kTile, 0, s>>>(B);
    k_batch_hop<REP, 3><<<grid, kTile, 0, s>>>(B);
    k_batch_xr<NC><<<grid, kTile, 0, s>>>(B);
    k_batch_p<NC><<<grid, kTile, 0, s>>>(B);
    return check_launch(ctx, "batched CG iteration");
}

// Device-side control of the one-graph batch solve: another pass of the WHILE
// body while some lattice is still iterating (its done flag also covers
// maxiter and NaN), at most 2 maxiter + 64 passes (counted in lattice 0's
// scalar block).
__global__ void k_batch_ctl(BatchArgs B, cudaGraphConditionalHandle h, int maxiter)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    bool all = true;
    for (int l = 0; l < B.nlat; ++l) all = all && sc(B.lat[l].scal, S_FLAGS, F_DONE) != 0.0;
    double &passes = sc(B.lat[0].scal, S_FLAGS, F_BODY);
    passes += 1.0;
    cudaGraphSetConditional(h, (!all && passes < 2.0 * maxiter + 64.0) ? 1u : 0u);
}

constexpr int kBatchIterPerPass = 8;

// The whole batched loop as one graph: a WHILE node whose body is
// kBatchIterPerPass iterations and the control kernel (iterations of
// converged lattices skip their tiles).
template <int REP>
hr_status capture_batch_while(hr_ctx *ctx, const BatchArgs &B, int grid, int maxiter, cudaGraph_t *out)
{
    cudaGraph_t G = nullptr;
    cudaStream_t cs = nullptr;
    bool capturing = false;
    hr_status st = HR_OK;
    cudaError_t e = cudaSuccess;
    auto fail = [&](const char *what) -> hr_status {
        if (capturing) {
            cudaGraph_t junk = nullptr;
            cudaStreamEndCapture(cs, &junk);
        }
        if (cs) cudaStreamDestroy(cs);
        if (G) cudaGraphDestroy(G);
        if (st) return st;
        return set_error(ctx, HR_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    };
    if ((e = cudaGraphCreate(&G, 0)) != cudaSuccess) return fail("graph create");
    if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) return fail("capture stream");
    cudaGraphConditionalHandle h;
    if ((e = cudaGraphConditionalHandleCreate(&h, G, 1, cudaGraphCondAssignDefault)) != cudaSuccess)
        return fail("loop condition");
    cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t wnode;
    if ((e = cudaGraphAddNode(&wnode, G, nullptr, nullptr, 0, &np)) != cudaSuccess) return fail("while node");
    cudaGraph_t body = np.conditional.phGraph_out[0];
    if ((e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
        cudaSuccess)
        return fail("begin capture");
    capturing = true;
    for (int k = 0; k < kBatchIterPerPass && !st; ++k) st = batch_launch_iteration<REP>(ctx, B, grid, cs);
    if (st) return fail("batched CG iteration");
    k_batch_ctl<<<1, 32, 0, cs>>>(B, h, maxiter);
    if ((st = check_launch(ctx, "batch control"))) return fail("batch control");
    cudaGraph_t same = nullptr;
    capturing = false;
    if ((e = cudaStreamEndCapture(cs, &same)) != cudaSuccess) return fail("end capture");
    cudaStreamDestroy(cs);
    *out = G;
    return HR_OK;
}

template <int REP>
hr_status batch_true_residual(hr_ctx *ctx, BatchArgs B, int grid, cudaStream_t s)
{
    constexpr int NC = RepTraits<REP>::NC;
    B.use_x = 1;
    B.ignore_done = 1;
    k_batch_hop<REP, 0><<<grid, kTile, 0, s>>>(B);
    k_batch_hop<REP, 1><<<grid, kTile, 0, s>>>(B);
    k_batch_hop<REP, 2><<<grid, kTile, 0, s>>>(B);
    k_batch_hop<REP, 3><<<grid, kTile, 0, s>>>(B);
    k_batch_residual<NC><<<grid, kTile, 0, s>>>(B);
    return check_launch(ctx, "batched true residual");
}

} // namespace

extern "C" {

size_t hr_cg_batch_workspace_bytes(int n_lat, const hr_lattice *lats, hr_rep rep)
{
    if (n_lat < 1 || n_lat > kMaxLattices || !lats || (rep != HR_FUND && rep != HR_ADJ)) return 0;
    for (int l = 0; l < n_lat; ++l)
        if (hr_spinor_packed_bytes(lats[l], rep, HR_F64, HR_EVEN, 1) == 0) return 0;
    return plan_batch(n_lat, lats, rep).bytes;
}

hr_status hr_cg_solve_batch(hr_ctx *ctx, int n_lat, const hr_lattice *lats, double m0, hr_rep rep,
                            const hr_solver_opts *opts, const void *const *gauges, const void *const *b,
                            void *const *x, hr_solve_info *infos, void *work, size_t work_bytes, hr_stream stream)
{
    if (!ctx) return HR_ERR_INVALID_ARG;
    if (n_lat < 1 || n_lat > kMaxLattices || !lats || !gauges || !b || !x)
        return set_error(ctx, HR_ERR_INVALID_ARG, "batch of 1..%d lattices with gauge, b and x arrays", kMaxLattices);
    if (rep != HR_FUND && rep != HR_ADJ)
        return set_error(ctx, HR_ERR_UNSUPPORTED, "batched solver: HR_FUND or HR_ADJ (quaternion links)");
    if (!opts || !(opts->tol > 0.0) || opts->maxiter < 1)
        return set_error(ctx, HR_ERR_INVALID_ARG, "tol must be > 0 and maxiter >= 1");
    if (opts->inner_prec != HR_F64 || opts->n_rhs != 1)
        return set_error(ctx, HR_ERR_UNSUPPORTED, "batched solver: FP64 CG with one RHS per lattice");
    if (!(4.0 + m0 != 0.0)) return set_error(ctx, HR_ERR_INVALID_ARG, "4 + m0 must be nonzero");
    for (int l = 0; l < n_lat; ++l) {
        hr_status st = validate_lattice(ctx, lats[l], 1);
        if (st) return st;
        if (make_geom(lats[l], 1).twisted)
            return set_error(ctx, HR_ERR_UNSUPPORTED, "batched solver: lattice %d has twisted boundaries", l);
        if (b[l] == x[l]) return set_error(ctx, HR_ERR_INVALID_ARG, "lattice %d: b and x alias", l);
        st = check_buffers(ctx, {gauges[l], b[l], x[l]});
        if (st) return st;
    }
    BatchPlan P = plan_batch(n_lat, lats, rep);
    if (!work || work_bytes < P.bytes)
        return set_error(ctx, HR_ERR_WORKSPACE, "workspace of %zu bytes needed, %zu given", P.bytes, work_bytes);
    if (hr_status sw = check_buffers(ctx, {work})) return sw;
    // values packed out of range since the last check (synchronises the stream)
    if (hr_status sp = consume_pack_status(ctx, (cudaStream_t)stream)) return sp;
    if (infos) std::memset(infos, 0, sizeof(hr_solve_info) * n_lat);
    cudaStream_t s = (cudaStream_t)stream;
    char *w = (char *)work;

    // descriptors and initial scalars
    const double A = 4.0 + m0;
    std::vector<BatchLat> desc(n_lat);
    std::vector<double> scal0(S_NSLOTS * kMaxRhsSlots, 0.0);
    scal0[S_ACTIVE * kMaxRhsSlots] = 1.0;
    scal0[S_DELTA2 * kMaxRhsSlots + 1] = opts->tol * opts->tol;
    scal0[S_DELTA2 * kMaxRhsSlots + 2] = opts->maxiter;
    int tile0 = 0;
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < n_lat; ++l) {
        BatchLat &L = desc[l];
        L.g = P.geoms[l];
        size_t h = spinor_half_bytes(L.g, rep, kF64);
        char *v = w + P.vec_off[l];
        L.gauge = gauges[l];
        L.b = b[l];
        L.x = x[l];
        L.r = v;
        L.p = v + h;
        L.q = v + 2 * h;
        L.u = v + 3 * h;
        L.t = v + 4 * h;
        L.scal = (double *)(w + P.scal_off[l]);
        L.partials = (double *)(w + P.part_off[l]);
        L.counters = (unsigned *)(w + P.cnt_off[l]);
        L.ntiles = (L.g.vh + kTile - 1) / kTile;
        L.tile0 = tile0;
        tile0 += L.ntiles;
        L.A = make_coef(A);
        L.negc = make_coef(-1.0 / (4.0 * A));
        if (e == cudaSuccess) e = cudaMemcpyAsync(L.scal, scal0.data(), sizeof(double) * scal0.size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(L.counters, 0, sizeof(unsigned) * kBatchCounters, s);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(w + P.desc_off, desc.data(), sizeof(BatchLat) * n_lat, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev0, s);
    if (e != cudaSuccess) return set_error(ctx, HR_ERR_CUDA, "batch set-up: %s", cudaGetErrorString(e));

    BatchArgs B;
    B.lat = (const BatchLat *)(w + P.desc_off);
    B.nlat = n_lat;
    B.total_tiles = P.total_tiles;
    B.use_x = 0;
    B.ignore_done = 0;
    B.unit = 1.f;
    B.nil = 0.f;
    int grid = ctx->sm_count > 0 ? ctx->sm_count * 8 : 1024;
    if (grid > P.total_tiles) grid = P.total_tiles;

    if (rep == HR_FUND) k_batch_start<2><<<grid, kTile, 0, s>>>(B);
    else k_batch_start<3><<<grid, kTile, 0, s>>>(B);
    hr_status st = check_launch(ctx, "batch start");
    if (st) return st;

    // check_every == 0: the whole loop is one graph (device-side WHILE);
    // check_every == N: a graph of N iterations, replayed with a host check after each
    const bool device_loop = opts->check_every <= 0;
    int chunk = device_loop ? kBatchIterPerPass : opts->check_every;
    if (chunk > opts->maxiter) chunk = opts->maxiter;
    GraphExec G;
    if (device_loop) {
        st = rep == HR_FUND ? capture_batch_while<kRepFund>(ctx, B, grid, opts->maxiter, &G.g)
                            : capture_batch_while<kRepAdj>(ctx, B, grid, opts->maxiter, &G.g);
        if (st) return st;
        e = cudaGraphInstantiate(&G.e, G.g, 0);
        if (e != cudaSuccess) return set_error(ctx, HR_ERR_CUDA, "batch graph: %s", cudaGetErrorString(e));
    } else {
        cudaStream_t cs;
        e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e != cudaSuccess) return set_error(ctx, HR_ERR_CUDA, "capture stream: %s", cudaGetErrorString(e));
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        for (int k = 0; k < chunk && e == cudaSuccess && !st; ++k)
            st = rep == HR_FUND ? batch_launch_iteration<kRepFund>(ctx, B, grid, cs)
                                : batch_launch_iteration<kRepAdj>(ctx, B, grid, cs);
        cudaError_t e2 = cudaStreamEndCapture(cs, &G.g);
        cudaStreamDestroy(cs);
        if (st) return st;
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&G.e, G.g, 0);
        if (e != cudaSuccess) return set_error(ctx, HR_ERR_CUDA, "batch graph: %s", cudaGetErrorString(e));
    }

    std::vector<double> flags((size_t)n_lat * kMaxRhsSlots);
    long long launched = 0;
    bool numeric = false;
    int max_iters = 0;
    for (;;) {
        e = cudaGraphLaunch(G.e, s);
        launched += chunk;
        for (int l = 0; l < n_lat && e == cudaSuccess; ++l)
            e = cudaMemcpyAsync(ctx->h_scal + (size_t)l * kMaxRhsSlots, desc[l].scal + S_FLAGS * kMaxRhsSlots,
                                sizeof(double) * kMaxRhsSlots, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return set_error(ctx, HR_ERR_CUDA, "batch iteration: %s", cudaGetErrorString(e));
        bool all = true;
        max_iters = 0;
        for (int l = 0; l < n_lat; ++l) {
            const double *f = ctx->h_scal + (size_t)l * kMaxRhsSlots;
            all = all && f[F_DONE] != 0.0;
            numeric = numeric || f[F_NUMERIC] != 0.0;
            if ((int)f[F_ITERS] > max_iters) max_iters = (int)f[F_ITERS];
        }
        if (device_loop || all || numeric || max_iters >= opts->maxiter || launched >= 2LL * opts->maxiter + chunk)
            break;
    }
    // true residuals
    st = rep == HR_FUND ? batch_true_residual<kRepFund>(ctx, B, grid, s) : batch_true_residual<kRepAdj>(ctx, B, grid, s);
    if (st) return st;
    e = cudaEventRecord(ctx->ev1, s);
    std::vector<double> host(S_NSLOTS * kMaxRhsSlots);
    bool all_ok = true;
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventSynchronize(ctx->ev1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    for (int l = 0; l < n_lat && e == cudaSuccess; ++l) {
        e = cudaMemcpy(host.data(), desc[l].scal, sizeof(double) * host.size(), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) break;
        double rr = host[S_OUT * kMaxRhsSlots], bb = host[S_BB * kMaxRhsSlots];
        double rel = bb > 0.0 ? std::sqrt(rr / bb) : 0.0;
        if (!std::isfinite(rel)) numeric = true;
        if (!(rel <= opts->tol)) all_ok = false;
        if (infos) {
            infos[l].iters = (int)host[S_FLAGS * kMaxRhsSlots + F_ITERS];
            infos[l].true_rel_residual = rel;
            infos[l].seconds = ms * 1e-3;
            infos[l].n_reliable_updates = 0;
        }
    }
    if (e != cudaSuccess) return set_error(ctx, HR_ERR_CUDA, "batch readback: %s", cudaGetErrorString(e));
    if (numeric) return set_error(ctx, HR_ERR_NUMERIC, "NaN or Inf in a batched CG residual");
    if (!all_ok) return set_error(ctx, HR_ERR_NOT_CONVERGED, "a lattice of the batch did not converge");
    return HR_OK;
}

} // extern "C"
