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
// position no polyhedral path diverges, so there is no tail hand-off: the
// paths are few compared with a total-degree homotopy of the same system.
#include "track_impl.cuh"

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
        const double2 c = tb.c1[q];
        const double p = __ldg(pw + q);
        double tp, dtp;  // t^p and p t^(p-1), with 0^0 = 1 (p >= 1 when p != 0)
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
        const double2 ct = make_double2(c.x * tp, c.y * tp);
        const double2 cr = dt ? make_double2(c.x * dtp, c.y * dtp) : ct;
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
                if (nx > o.diverge_norm) {
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

cudaError_t launch_track_poly(const PolyLaunch &L, int block_threads, int max_blocks, cudaStream_t s)
{
    device_limits();
    if (L.n_paths <= 0) return cudaSuccess;
#define PHC_CALL_TP(NN) launch_track_poly_n<NN>(L, block_threads, max_blocks, s)
    PHC_DISPATCH_N(L.tab.n, PHC_CALL_TP)
#undef PHC_CALL_TP
}

}  // namespace phc
