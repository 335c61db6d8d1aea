// track_poly.cu -- polyhedral homotopies (Section 2.2) on the GPU: the start
// solutions of every mixed cell's binomial system, and the paths from them to
// the roots of the random coefficient system g.
//
// Path p of a polyhedral handle belongs to the cell whose range of paths
// holds it (binary search over the cells' first paths).  Its start solution
// comes from the cell's Hermite form U D = H: with beta_j = -c_{a_j} / c_{b_j}
// and the digits r_k of p's index within the cell in the radices H_kk,
//   log y_k = (sum_j U_kj log beta_j - sum_{l>k} H_kl log y_l + 2 pi i r_k) / H_kk
// for k = n-1 .. 0, so that y^{H_k} = prod_j beta_j^{U_kj} (every branch of
// the logarithms gives a solution, and the digits run through all |det D|).
// The cell's homotopy is sum_q c_q t^{p_q} y^{a_q} with per-cell powers p_q
// (0 on the cell's terms, >= 1 elsewhere): the evaluation is track_kernel's
// Speelpenning evaluation (add_term) with the coefficient c_q t^{p_q} in H
// and H_x and c_q p_q t^{p_q - 1} in H_t.  One thread per path with the
// step logic of track_kernel's readings (RK4 predictor, Newton corrector,
// step control, end Newton at t = 1); classification in classify_kernel at
// t = 1, where every cell's homotopy is g.  For coefficients in general
// position no polyhedral path diverges, and the paths are few compared with a
// total-degree homotopy of the same system: a launch whose paths fit in one
// wave of groups runs a group of lanes per path instead (poly_group_kernel,
// the tail kernels' tail_path), with the same results bit for bit.
#include "tail_impl.cuh"

namespace phc {

#define PHC_TWO_PI 6.283185307179586476925286766559

// Start solution of global path gid; returns its cell.
template <int N>
__device__ int poly_start(const PolyLaunch &L, int64_t gid, double2 (&y)[N])
{
    int lo = 0, hi = L.n_cells - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (L.path_off[mid] <= gid) lo = mid;
        else hi = mid - 1;
    }
    const int cell = lo;
    int64_t r = gid - L.path_off[cell];
    const int64_t *H = L.H + (size_t)cell * N * N;
    const int64_t *U = L.U + (size_t)cell * N * N;
    const int32_t *pr = L.pairs + (size_t)cell * 2 * N;
    double2 lb[N];
#pragma unroll
    for (int j = 0; j < N; j++) {
        const double2 ca = L.tab.c1[pr[2 * j]], cb = L.tab.c1[pr[2 * j + 1]];
        // beta = -ca / cb
        const double2 q = cmul(make_double2(-ca.x, -ca.y), recip(cb));
        lb[j] = make_double2(log(hypot(q.x, q.y)), atan2(q.y, q.x));
    }
    int64_t digit[N];
#pragma unroll
    for (int k = 0; k < N; k++) {
        const int64_t d = H[k * N + k];
        digit[k] = r % d;
        r /= d;
    }
    double2 ly[N];
#pragma unroll
    for (int k = N - 1; k >= 0; k--) {
        double sx = 0.0, sy = 0.0;
#pragma unroll
        for (int j = 0; j < N; j++) {
            const double u = (double)U[k * N + j];
            sx = fma(u, lb[j].x, sx);
            sy = fma(u, lb[j].y, sy);
        }
#pragma unroll
        for (int l = k + 1; l < N; l++) {
            const double hk = (double)H[k * N + l];
            sx = fma(-hk, ly[l].x, sx);
            sy = fma(-hk, ly[l].y, sy);
        }
        sy = fma(PHC_TWO_PI, (double)digit[k], sy);
        const double d = (double)H[k * N + k];
        ly[k] = make_double2(sx / d, sy / d);
    }
#pragma unroll
    for (int k = 0; k < N; k++) {
        double s, c;
        sincos(ly[k].y, &s, &c);
        const double m = exp(ly[k].x);
        y[k] = make_double2(m * c, m * s);
    }
    return cell;
}

template <int N>
__global__ void __launch_bounds__(256) poly_starts_kernel(const PolyLaunch L)
{
    const int64_t np = L.n_paths, xld = L.x_ld ? L.x_ld : np;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < np; q += (int64_t)gridDim.x * blockDim.x) {
        double2 y[N];
        poly_start<N>(L, L.first + q, y);
#pragma unroll
        for (int j = 0; j < N; j++) L.x_out[(int64_t)j * xld + q] = y[j];
    }
}

// Term q's coefficient in the cell's homotopy at t: c t^p in H and H_x, and
// in the right-hand side c p t^(p-1) (H_t, dt) or c t^p (H); 0^0 = 1 and
// p >= 1 when p != 0; lt = log t (unused at t = 0).
__device__ __forceinline__ void poly_coef(double2 c, double p, double t, double lt, bool dt, double2 &ct, double2 &cr)
{
    double tp, dtp;
    if (p == 0.0) {
        tp = 1.0;
        dtp = 0.0;
    } else if (t == 0.0) {
        tp = 0.0;
        dtp = p == 1.0 ? 1.0 : 0.0;
    } else {
        tp = exp(p * lt);
        dtp = p * tp / t;
    }
    ct = make_double2(c.x * tp, c.y * tp);
    cr = dt ? make_double2(c.x * dtp, c.y * dtp) : ct;
}

// Divergence bound of a polyhedral path: diverge_norm x max(1, ||y(0)||).
// The start solution of a cell's binomial system (the y coordinates at t = 0)
// may itself lie beyond diverge_norm without the path diverging.
template <int N>
__device__ __forceinline__ double poly_diverge_bound(const double2 (&y)[N], double diverge_norm)
{
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < N; j++) {
        const double a = absinf(y[j]);
        if (!(a <= s)) s = a;
    }
    return diverge_norm * (s > 1.0 ? s : 1.0);
}

// The same coefficients for tail_path (the grouped tracker), log t taken
// once per t; div: the path's divergence bound.
struct PolyCoef {
    const double2 *C;
    const double *pw;
    double last_t, lt, div;
    __device__ __forceinline__ double diverge_bound(const phc_opts &) const { return div; }
    __device__ __forceinline__ void operator()(int q, double te, bool dt, double2 &ct, double2 &cr)
    {
        if (te != last_t) {
            last_t = te;
            lt = te > 0.0 ? log(te) : 0.0;
        }
        poly_coef(C[q], __ldg(pw + q), te, lt, dt, ct, cr);
    }
};

// J = H_x (row-major N x N) and R = H_t (dt) or H (!dt) at (X, t) for the
// cell's homotopy sum_q c_q t^{p_q} y^{a_q}; lt = log t (unused at t = 0).
template <int N>
__device__ __forceinline__ void evaluate_poly(const SmTab &tb, const double *pw, double t, double lt, bool dt,
                                              const double2 *X, double2 *R, double2 *J, int bt)
{
    const double2 zero = make_double2(0.0, 0.0);
#pragma unroll
    for (int i = 0; i < N; i++) st(R, i, bt, zero);
#pragma unroll
    for (int i = 0; i < N * N; i++) st(J, i, bt, zero);
    for (int q = 0; q < tb.n_terms; q++) {
        const TermRec r = tb.terms[q];
        double2 ct, cr;
        poly_coef(tb.c1[q], __ldg(pw + q), t, lt, dt, ct, cr);
        if (r.k == 0) {
            st(R, r.eq, bt, cadd(ld<double2>(R, r.eq, bt), cr));
            continue;
        }
        AccumSink<double2, true, N> sink{J + r.eq * N * bt, R + r.eq * bt, nullptr, bt, true, {}};
        add_term<double2>(r, tb.vars + r.off, tb.exps + r.off, ct, cr, X, bt, sink);
    }
}

// Solves J d = R in place (R := d); false on a zero pivot.
template <int N>
__device__ __forceinline__ bool solve_poly(double2 *J, double2 *R, int bt)
{
    int perm[N];
    if (!lu_factor<N, double2>(J, perm, bt)) return false;
    lu_solve<N, double2>(J, perm, R, bt);
    return true;
}

// Max-norm of the correction in R and of x - correction, written back to xe.
template <int N>
__device__ __forceinline__ bool newton_update(double2 *xe, const double2 *R, int bt, double *d_out, double *nx_out,
                                              double2 (*keep)[N])
{
    double d = 0.0, nx = 0.0;
    bool fin = true;
#pragma unroll
    for (int j = 0; j < N; j++) {
        const double2 dj = ld<double2>(R, j, bt);
        const double2 xo = ld<double2>(xe, j, bt);
        const double2 xj = make_double2(xo.x - dj.x, xo.y - dj.y);
        st(xe, j, bt, xj);
        if (keep) (*keep)[j] = xj;
        const double a = absinf(dj);
        if (!(a <= d)) d = a;
        const double b = absinf(xj);
        if (!(b <= nx)) nx = b;
        fin = fin && finite2(xj);
    }
    *d_out = d;
    *nx_out = nx;
    return fin;
}

template <int N>
__global__ void __launch_bounds__(256) track_poly_kernel(const PolyLaunch L, size_t table_bytes)
{
    extern __shared__ __align__(16) char smem[];
    const SmTab tb = stage_table(L.tab, smem);
    const int bt = blockDim.x;
    double2 *xe = reinterpret_cast<double2 *>(smem + table_bytes) + threadIdx.x;
    double2 *R = xe + N * bt;
    double2 *J = R + N * bt;
    const phc_opts &o = L.o;
    const int64_t np = L.n_paths, xld = L.x_ld ? L.x_ld : np;
    double2 x0[N], acc[N];
    for (;;) {
        const unsigned long long c = atomicAdd(L.qhead, 1ull);
        if (c >= (unsigned long long)np) break;
        const int64_t q = (int64_t)c;
        const int cell = poly_start<N>(L, L.first + q, x0);
        const double *pw = L.powers + (size_t)cell * tb.n_terms;
        const double div = poly_diverge_bound<N>(x0, o.diverge_norm);
        double t = 0.0, h = o.h_init, next_s = 0.1;
        double r0 = 0.0, r1 = 0.0, r2 = 0.0, r3 = 0.0, r4 = 0.0;
        int streak = 0, steps = 0, nck = 0, since_ck = 0, n_acc = 0, n_rej = 0, n_newt = 0, n_solve = 0;
        int stop = -1;
        // ------------------------------------------------------------ steps
        while (stop < 0) {
            double he = h, t1 = t + he;
            if (he >= 1.0 - t) {
                he = 1.0 - t;
                t1 = 1.0;
            }
            bool ok = true;
            // predictor: RK4, k_s = -J^{-1} H_t at the stage points
#pragma unroll
            for (int j = 0; j < N; j++) st(xe, j, bt, x0[j]);
            for (int stage = 0; stage < 4 && ok; stage++) {
                const double ts = stage == 0 ? t : stage < 3 ? t + 0.5 * he : t1;
                evaluate_poly<N>(tb, pw, ts, ts > 0.0 ? log(ts) : 0.0, true, xe, R, J, bt);
                n_solve++;
                ok = solve_poly<N>(J, R, bt);
                if (!ok) break;
#pragma unroll
                for (int j = 0; j < N; j++) {
                    const double2 k = ld<double2>(R, j, bt);
                    const double2 kj = make_double2(-k.x, -k.y);
                    acc[j] = stage == 0 ? kj : caxpy(acc[j], stage == 3 ? 1.0 : 2.0, kj);
                    if (stage < 2) st(xe, j, bt, caxpy(x0[j], 0.5 * he, kj));
                    else if (stage == 2) st(xe, j, bt, caxpy(x0[j], he, kj));
                }
            }
            if (ok) {
#pragma unroll
                for (int j = 0; j < N; j++) st(xe, j, bt, caxpy(x0[j], he / 6.0, acc[j]));
            }
            // corrector: Newton at t1
            bool conv = false;
            double prev = 0.0;
            const double lt1 = log(t1);
            for (int it = 0; ok && it < o.max_corr_iters; it++) {
                evaluate_poly<N>(tb, pw, t1, lt1, false, xe, R, J, bt);
                n_solve++;
                n_newt++;
                if (!solve_poly<N>(J, R, bt)) break;
                double d, nx;
                const bool fin = newton_update<N>(xe, R, bt, &d, &nx, nullptr);
                if (!(d == d) || !fin) break;
                if (d <= o.corr_tol * (1.0 + nx)) {
                    conv = true;
                    break;
                }
                if (it > 0 && d > o.corr_contract * prev) break;
                prev = d;
            }
            steps++;
            if (conv) {
                t = t1;
                double nx = 0.0;
#pragma unroll
                for (int j = 0; j < N; j++) {
                    x0[j] = ld<double2>(xe, j, bt);
                    const double a = absinf(x0[j]);
                    if (!(a <= nx)) nx = a;
                }
                n_acc++;
                while (1.0 - t <= next_s && next_s > 0.0) {
                    r0 = r1;
                    r1 = r2;
                    r2 = r3;
                    r3 = r4;
                    r4 = nx;
                    nck++;
                    since_ck = 0;
                    next_s *= 0.1;
                    if (nck >= 40) next_s = 0.0;
                }
                if (nx > div) {
                    stop = PHC_STOP_DIVERGED;
                    break;
                }
                if (++streak >= o.expand_after) {
                    streak = 0;
                    h = h * o.expand;
                    if (h > o.h_max) h = o.h_max;
                }
            } else {
                n_rej++;
                streak = 0;
                h = he * o.shrink;
                if (h < o.h_min) {
                    stop = PHC_STOP_STEP_MIN;
                    break;
                }
            }
            if (steps >= o.max_steps) stop = PHC_STOP_BUDGET;
            else if (++since_ck >= o.max_steps_decade && t < 1.0) stop = PHC_STOP_BUDGET;
            else if (t >= 1.0) stop = PHC_STOP_REACHED;
        }
        // ------------------------------------------------------------ end Newton at t = 1
        if (stop == PHC_STOP_REACHED) {
#pragma unroll
            for (int j = 0; j < N; j++) st(xe, j, bt, x0[j]);
            for (int it = 0; it < o.end_iters; it++) {
                evaluate_poly<N>(tb, pw, 1.0, 0.0, false, xe, R, J, bt);
                n_solve++;
                n_newt++;
                if (!solve_poly<N>(J, R, bt)) break;
                double d, nx;
                const bool fin = newton_update<N>(xe, R, bt, &d, &nx, &x0);
                if (!(d == d) || !fin) break;
                if (d <= o.end_tol * (1.0 + nx)) break;
            }
        }
        int grew = 0;
        double growth = 0.0;
        if (nck >= 2) {
            const int l = nck - 1, m = l < 4 ? l : 4;
            const double a = r4, b = (m == 1) ? r3 : (m == 2) ? r2 : (m == 3) ? r1 : r0;
            double g = 1.0;
            for (int k = 0; k < m; k++) g *= o.growth_inf;
            grew = a > b * g;
            growth = log10(a / b) / m;
        }
        phc_path_stats rec;
        rec.t = t;
        rec.h = h;
        rec.cond = 0.0;
        rec.relres = 0.0;
        rec.norm_x = 0.0;
        rec.growth = growth;
        rec.n_accept = n_acc;
        rec.n_reject = n_rej;
        rec.n_newton = n_newt;
        rec.n_solve = n_solve;
        rec.stop = stop;
        rec.n_fp32 = 0;
        rec.grew = grew;
        rec.system = 0;
#pragma unroll
        for (int j = 0; j < N; j++) L.x_out[(int64_t)j * xld + q] = x0[j];
        L.stats[q] = rec;
    }
}

// A group of G lanes per path (tail_path of tail_impl.cuh with the cell's
// coefficients): the same operations in the same order as track_poly_kernel,
// at a fraction of the latency per unit, for launches of few paths.
template <int N, int G>
__global__ void __launch_bounds__(128) poly_group_kernel(const PolyLaunch L, size_t table_bytes, size_t plan_bytes)
{
    extern __shared__ __align__(16) char smem[];
    const SmTab tb = stage_table(L.tab, smem);
    const TailPlan plan = plan_layout<N>(tb, smem + table_bytes);
    if (threadIdx.x == 0) plan_fill<N>(tb, plan);
    __syncthreads();
    const int S = tail_store_slots(tb.n_terms, L.tab.n_ve);
    const int lane = threadIdx.x & 31;
    const int r = lane % G;  // the row this lane owns in the LU and the solves (r < N)
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane - r));
    const int group = threadIdx.x / G;
    double2 *base = reinterpret_cast<double2 *>(smem + table_bytes + plan_bytes) +
                    (size_t)group * tail_group_slots(N, S);
    const int64_t np = L.n_paths, xld = L.x_ld ? L.x_ld : np;
    for (;;) {
        unsigned long long c = 0;
        if (r == 0) c = atomicAdd(L.qhead, 1ull);
        c = __shfl_sync(gmask, c, 0, G);
        if (c >= (unsigned long long)np) break;
        const int64_t q = (int64_t)c;
        // a fresh path: t = 0 at the cell's binomial solution
        Handoff hd;
        double2 y[N];
        const int cell = poly_start<N>(L, L.first + q, y);
#pragma unroll
        for (int j = 0; j < N; j++) hd.x0[j] = y[j];
        hd.t = 0.0;
        hd.h = L.o.h_init;
        hd.next_s = 0.1;
        hd.nx0 = hd.r0 = hd.r1 = hd.r2 = hd.r3 = hd.r4 = 0.0;
        hd.q = q;
        hd.sys = hd.streak = hd.steps = hd.since_ck = hd.nck = 0;
        hd.n_acc = hd.n_rej = hd.n_newt = hd.n_solve = hd.n_f32 = hd.stage = 0;
        const PolyCoef coef{tb.c1, L.powers + (size_t)cell * tb.n_terms, -1.0, 0.0,
                            poly_diverge_bound<N>(y, L.o.diverge_norm)};
        tail_path<N, G>(hd, tb, plan, coef, base, L.o, r, gmask, [&](double2 x0r, const phc_path_stats &rec, int) {
            if (r < N) L.x_out[(int64_t)r * xld + q] = x0r;
            if (r == 0) L.stats[q] = rec;
        });
    }
}

template <int N>
static cudaError_t launch_poly_starts_n(const PolyLaunch &L, cudaStream_t s)
{
    int64_t grid = (L.n_paths + 127) / 128;
    if (grid > (int64_t)g_num_sms * 16) grid = (int64_t)g_num_sms * 16;
    if (grid < 1) grid = 1;
    poly_starts_kernel<N><<<(unsigned)grid, 128, 0, s>>>(L);
    return cudaGetLastError();
}

cudaError_t launch_poly_starts(const PolyLaunch &L, cudaStream_t s)
{
    device_limits();
    if (L.n_paths <= 0) return cudaSuccess;
#define PHC_CALL_PS(NN) launch_poly_starts_n<NN>(L, s)
    PHC_DISPATCH_N(L.tab.n, PHC_CALL_PS)
#undef PHC_CALL_PS
}

template <int N>
static cudaError_t launch_track_poly_n(const PolyLaunch &L, int block_threads, int max_blocks, cudaStream_t s)
{
    const size_t tb = table_smem_bytes(L.tab);
    const int bt = track_block_threads(N, tb, block_threads, false, false, true);
    if (bt == 0) return cudaErrorInvalidConfiguration;
    const size_t smem = tb + (size_t)bt * thread_smem_bytes(N, false, false, true);
    cudaError_t e = cudaFuncSetAttribute(track_poly_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, track_poly_kernel<N>, bt, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int64_t want = (L.n_paths + bt - 1) / bt;
    int64_t grid = (int64_t)g_num_sms * per_sm;
    if (max_blocks > 0 && grid > max_blocks) grid = max_blocks;
    if (grid > want) grid = want;
    if (grid < 1) grid = 1;
    track_poly_kernel<N><<<(unsigned)grid, bt, smem, s>>>(L, tb);
    return cudaGetLastError();
}

// The grouped launch: groups of G lanes in blocks of up to 128 threads, as
// many blocks as are resident; *capacity = the groups resident at once (the
// paths one wave takes).  launch = false only computes the capacity.
template <int N, int G>
static cudaError_t launch_poly_group_n(const PolyLaunch &L_in, int max_blocks, cudaStream_t s, bool launch,
                                       int64_t *capacity)
{
    PolyLaunch L = L_in;
    L.tab.coef_smem = 1;
    size_t tb = table_smem_bytes(L.tab);
    const size_t pb = tail_plan_bytes(N, L.tab.n_terms, L.tab.n_ve);
    const size_t per_group = (size_t)tail_group_slots(N, tail_store_slots(L.tab.n_terms, L.tab.n_ve)) * sizeof(double2);
    int groups = 128 / G;
    if (tb + pb + groups * per_group > (size_t)g_smem_optin) {
        L.tab.coef_smem = 0;  // coefficients through L1
        tb = table_smem_bytes(L.tab);
    }
    while (groups > 1 && tb + pb + groups * per_group > (size_t)g_smem_optin) groups /= 2;
    const size_t smem = tb + pb + groups * per_group;
    if (smem > (size_t)g_smem_optin) return cudaErrorInvalidConfiguration;
    const int bt = groups * G;
    cudaError_t e = cudaFuncSetAttribute(poly_group_kernel<N, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, poly_group_kernel<N, G>, bt, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int64_t grid = (int64_t)g_num_sms * per_sm;
    if (max_blocks > 0 && grid > max_blocks) grid = max_blocks;
    *capacity = grid * groups;
    if (!launch) return cudaSuccess;
    const int64_t want = (L.n_paths + groups - 1) / groups;
    if (grid > want) grid = want;
    if (grid < 1) grid = 1;
    poly_group_kernel<N, G><<<(unsigned)grid, bt, smem, s>>>(L, tb, pb);
    return cudaGetLastError();
}

template <int N>
static cudaError_t launch_poly_group_g(const PolyLaunch &L, int group, int max_blocks, cudaStream_t s, bool launch,
                                       int64_t *capacity)
{
    if (group == 8 && N <= 8) return launch_poly_group_n<N, (N <= 8 ? 8 : 16)>(L, max_blocks, s, launch, capacity);
    if (group == 16) return launch_poly_group_n<N, 16>(L, max_blocks, s, launch, capacity);
    return launch_poly_group_n<N, 32>(L, max_blocks, s, launch, capacity);
}

// opts.group_paths: 1 a group per path, -1 one thread per path, 0 a group
// per path unless the paths exceed 32 waves of the resident groups.  A group
// runs a unit several times faster than one thread (the latency of the
// longest paths sets the time of a launch of few paths), and measured faster
// at every size tried (random cyclic 7 .. 10, 924 to 35,940 paths: 15 against
// 95 ms, 20 against 94, 97 against 193, 546 against 610).  The group has
// opts.tail_threads lanes, or by default 32 for N <= 7 and 16 above (the
// faster of the two on those systems).
cudaError_t launch_track_poly(const PolyLaunch &L, int block_threads, int max_blocks, cudaStream_t s)
{
    device_limits();
    if (L.n_paths <= 0) return cudaSuccess;
    const int gp = L.o.group_paths;
    const int group = L.o.tail_threads ? L.o.tail_threads : (L.tab.n <= 7 ? 32 : 16);
    const bool fits = tail_supported(L.tab);
    bool grouped = gp == 1 && fits;
    if (gp == 0 && fits) {
        int64_t cap = 0;
        cudaError_t e = cudaErrorInvalidValue;
#define PHC_CALL_CAP(NN) launch_poly_group_g<NN>(L, group, max_blocks, s, false, &cap)
        switch (L.tab.n) {
        case 1: e = PHC_CALL_CAP(1); break;
        case 2: e = PHC_CALL_CAP(2); break;
        case 3: e = PHC_CALL_CAP(3); break;
        case 4: e = PHC_CALL_CAP(4); break;
        case 5: e = PHC_CALL_CAP(5); break;
        case 6: e = PHC_CALL_CAP(6); break;
        case 7: e = PHC_CALL_CAP(7); break;
        case 8: e = PHC_CALL_CAP(8); break;
        case 9: e = PHC_CALL_CAP(9); break;
        case 10: e = PHC_CALL_CAP(10); break;
        case 11: e = PHC_CALL_CAP(11); break;
        case 12: e = PHC_CALL_CAP(12); break;
        default: break;
        }
#undef PHC_CALL_CAP
        grouped = e == cudaSuccess && L.n_paths <= 32 * cap;
    }
    if (grouped) {
        int64_t cap = 0;
#define PHC_CALL_TG(NN) launch_poly_group_g<NN>(L, group, max_blocks, s, true, &cap)
        PHC_DISPATCH_N(L.tab.n, PHC_CALL_TG)
#undef PHC_CALL_TG
    }
#define PHC_CALL_TP(NN) launch_track_poly_n<NN>(L, block_threads, max_blocks, s)
    PHC_DISPATCH_N(L.tab.n, PHC_CALL_TP)
#undef PHC_CALL_TP
}

}  // namespace phc
