// endgame.cu -- the Cauchy endgame for singular endpoints.
//
// A path of the total-degree homotopy that converges to a singular endpoint
// x* has, near t = 1, an expansion x(s) = x* + sum_k a_k s^{k/c} in
// s = 1 - t, with c the cycle number (a double root met by two paths gives
// c = 2).  The tracker's Newton steps at t = 1 converge only linearly there
// and leave x* accurate to about the square root of the unit roundoff.  The
// endgame tracks the path to t0 = 1 - EG_RADIUS, then around the circle
// s = EG_RADIUS e^{i theta} in complex t until the path closes up after c
// loops, sampling x at EG_SAMPLES equally spaced angles per loop.  By
// Cauchy's integral formula in the variable s^{1/c}, the mean of the
// c * EG_SAMPLES samples is x* (the trapezoidal rule on a closed loop, exact
// up to terms of order EG_RADIUS^EG_SAMPLES).  A path that runs to infinity
// closes up too (a pole in s) but its mean is no root: an estimate counts only
// when its relative residual max_i |H_i(x*, 1)|_1 / (1 + scale_i) is at most
// EG_RES.  One thread per path; the evaluation and LU are the tracker's
// (add_term, lu_factor, lu_solve) with the coefficient c0 + t c1 at a complex t.
#include "track_impl.cuh"

namespace phc {

#define EG_RADIUS 0.01
#define EG_SAMPLES 16
#define EG_MAX_CYCLES 8
#define EG_CLOSE_TOL 1e-8
#define EG_RES 1e-10

// J = H_x and R = H_t (dt) or H (!dt) at (X, tc), tc complex.
template <int N>
__device__ __forceinline__ void evaluate_ct(const double2 *C0, const double2 *C1, const SmTab &tb, double2 tc, bool dt,
                                            const double2 *X, double2 *R, double2 *J, double2 *P, int bt)
{
    const double2 zero = make_double2(0.0, 0.0);
#pragma unroll
    for (int i = 0; i < N; i++) SL(R, i) = zero;
#pragma unroll
    for (int i = 0; i < N * N; i++) SL(J, i) = zero;
    for (int q = 0; q < tb.n_terms; q++) {
        const TermRec r = tb.terms[q];
        const double2 c0 = C0[q], c1 = C1[q];
        const double2 ct = cfma(tc, c1, c0);
        const double2 cr = dt ? c1 : ct;
        if (r.k == 0) {
            SL(R, r.eq) = cadd(SL(R, r.eq), cr);
            continue;
        }
        AccumSink<double2> sink{J + r.eq * N * bt, R + r.eq * bt, P, bt, true, {}};
        add_term<double2>(r, tb.vars + r.off, tb.exps + r.off, ct, cr, X, bt, sink);
    }
}

// Solves J y = R (R := y) after evaluate_ct; false on a zero pivot.
template <int N>
__device__ __forceinline__ bool solve_ct(double2 *J, double2 *R, int bt)
{
    int perm[N];
    if (!lu_factor<N, double2>(J, perm, bt)) return false;
    lu_solve<N, double2>(J, perm, R, bt);
    return true;
}

__device__ __forceinline__ double norm_n(const double2 *v, int n)
{
    double m = 0.0;
    for (int j = 0; j < n; j++) {
        const double a = absinf(v[j]);
        if (!(a <= m)) m = a;
    }
    return m;
}

template <int N>
__global__ void __launch_bounds__(128) endgame_kernel(const TrackLaunch L, size_t table_bytes, int32_t *cycle_out)
{
    extern __shared__ __align__(16) char smem[];
    const SmTab tb = stage_table(L.tab, smem);
    const int bt = blockDim.x;
    double2 *xe = reinterpret_cast<double2 *>(smem + table_bytes) + threadIdx.x;
    double2 *R = xe + N * bt, *P = R + N * bt, *J = P + N * bt, *S = J + N * N * bt;
    const phc_opts &o = L.o;
    const int64_t np = L.n_paths;
    const double t0 = 1.0 - EG_RADIUS;
    double2 x[N], x0[N], acc[N];
    for (;;) {
        const unsigned long long cq = atomicAdd(L.qhead, 1ull);
        if (cq >= (unsigned long long)np) break;
        const int64_t q = (int64_t)cq;
        const int64_t gid = L.first + q;
        const int sys = (int)(gid / L.paths_per_system);
        int64_t pid = gid - (int64_t)sys * L.paths_per_system;
        for (int i = 0; i < N; i++) {
            const int d = L.deg[i];
            const int k = (int)(pid % d);
            pid /= d;
            x[i] = L.roots[L.root_off[i] + k];
        }
        const double2 *C0 = tb.c0 + (size_t)sys * tb.n_terms, *C1 = tb.c1 + (size_t)sys * tb.n_terms;
        phc_path_stats rec = {};
        rec.system = sys;
        int stop = 0, cycle = 0;
        // one Runge-Kutta + Newton step of size he from (x, p) along the real t
        // segment (circle = false) or the circle (circle = true: p is the angle);
        // returns whether the corrector converged (x holds the new point then)
        auto step = [&](double p, double he, bool circle) -> bool {
#pragma unroll
            for (int j = 0; j < N; j++) x0[j] = x[j];
            bool ok = true;
            for (int stg = 0; stg < 4 && ok; stg++) {
                const double ps = stg == 0 ? p : stg < 3 ? p + 0.5 * he : p + he;
                double2 tc, dtdp;
                if (circle) {
                    double sn, cs;
                    sincos(ps, &sn, &cs);
                    tc = make_double2(1.0 - EG_RADIUS * cs, -EG_RADIUS * sn);
                    dtdp = make_double2(EG_RADIUS * sn, -EG_RADIUS * cs);  // -i r e^{i theta}
                } else {
                    tc = make_double2(ps, 0.0);
                    dtdp = make_double2(1.0, 0.0);
                }
                for (int j = 0; j < N; j++) SL(xe, j) = stg == 0 ? x0[j] : SL(xe, j);
                evaluate_ct<N>(C0, C1, tb, tc, true, xe, R, J, P, bt);
                rec.n_solve++;
                ok = solve_ct<N>(J, R, bt);
                if (!ok) break;
                const double w = (stg == 0 || stg == 3) ? 1.0 : 2.0;
                const double hs = stg < 2 ? 0.5 * he : he;
#pragma unroll
                for (int j = 0; j < N; j++) {
                    const double2 v = cmul(SL(R, j), dtdp);
                    const double2 kj = make_double2(-v.x, -v.y);
                    acc[j] = stg == 0 ? kj : caxpy(acc[j], w, kj);
                    if (stg < 3) SL(xe, j) = caxpy(x0[j], hs, kj);
                }
            }
            if (!ok) return false;
#pragma unroll
            for (int j = 0; j < N; j++) SL(xe, j) = caxpy(x0[j], he / 6.0, acc[j]);
            double2 tc;
            if (circle) {
                double sn, cs;
                sincos(p + he, &sn, &cs);
                tc = make_double2(1.0 - EG_RADIUS * cs, -EG_RADIUS * sn);
            } else {
                tc = make_double2(p + he, 0.0);
            }
            double prev = 0.0;
            for (int it = 0; it < o.max_corr_iters; it++) {
                evaluate_ct<N>(C0, C1, tb, tc, false, xe, R, J, P, bt);
                rec.n_solve++;
                rec.n_newton++;
                if (!solve_ct<N>(J, R, bt)) return false;
                double d = 0.0, nx = 0.0;
                bool fin = true;
                for (int j = 0; j < N; j++) {
                    const double2 dj = SL(R, j);
                    const double2 xj = make_double2(SL(xe, j).x - dj.x, SL(xe, j).y - dj.y);
                    SL(xe, j) = xj;
                    const double a = absinf(dj);
                    if (!(a <= d)) d = a;
                    const double b = absinf(xj);
                    if (!(b <= nx)) nx = b;
                    fin = fin && finite2(xj);
                }
                if (!(d == d) || !fin) return false;
                if (d <= o.corr_tol * (1.0 + nx)) {
                    for (int j = 0; j < N; j++) x[j] = SL(xe, j);
                    return true;
                }
                if (it > 0 && d > o.corr_contract * prev) return false;
                prev = d;
            }
            return false;
        };
        // ---------------------------------------------------- along t to t0
        double t = 0.0, h = o.h_init;
        int streak = 0, steps = 0;
        while (t < t0) {
            double he = h, t1 = t + he;
            if (he >= t0 - t) {
                he = t0 - t;
                t1 = t0;
            }
            steps++;
            if (step(t, he, false)) {
                t = t1;
                rec.n_accept++;
                if (norm_n(x, N) > o.diverge_norm) {
                    stop = PHC_STOP_DIVERGED;
                    break;
                }
                if (++streak >= o.expand_after) {
                    streak = 0;
                    h = h * o.expand;
                    if (h > o.h_max) h = o.h_max;
                }
            } else {
                for (int j = 0; j < N; j++) x[j] = x0[j];
                rec.n_reject++;
                streak = 0;
                h = he * o.shrink;
                if (h < o.h_min) {
                    stop = PHC_STOP_STEP_MIN;
                    break;
                }
            }
            if (steps >= o.max_steps) {
                stop = PHC_STOP_BUDGET;
                break;
            }
        }
        rec.t = t;
        // ---------------------------------------------------- around the circle
        if (stop == 0 && t >= t0) {
            const double dth = 2.0 * 3.141592653589793 / EG_SAMPLES, hmin = dth * 9.5367431640625e-07;  // 2^-20
            double2 start[N], sum[N];
            for (int j = 0; j < N; j++) {
                start[j] = x[j];
                sum[j] = make_double2(0.0, 0.0);
            }
            double th = 0.0, hth = dth;
            streak = 0;
            bool failed = false;
            for (int sample = 1; sample <= EG_SAMPLES * EG_MAX_CYCLES && !failed && !cycle; sample++) {
                for (int j = 0; j < N; j++) sum[j] = cadd(sum[j], x[j]);
                const double target = sample * dth;
                while (th < target) {
                    double he = hth, t1 = th + he;
                    if (he >= target - th) {
                        he = target - th;
                        t1 = target;
                    }
                    if (step(th, he, true)) {
                        th = t1;
                        rec.n_accept++;
                        if (++streak >= o.expand_after) {
                            streak = 0;
                            hth = hth * o.expand;
                            if (hth > dth) hth = dth;
                        }
                    } else {
                        for (int j = 0; j < N; j++) x[j] = x0[j];
                        rec.n_reject++;
                        streak = 0;
                        hth = he * o.shrink;
                        if (hth < hmin) {
                            failed = true;
                            stop = PHC_STOP_STEP_MIN;
                            break;
                        }
                    }
                }
                if (!failed && sample % EG_SAMPLES == 0) {
                    double d = 0.0;
                    for (int j = 0; j < N; j++) {
                        const double a = absinf(make_double2(x[j].x - start[j].x, x[j].y - start[j].y));
                        if (!(a <= d)) d = a;
                    }
                    if (d <= EG_CLOSE_TOL * (1.0 + norm_n(start, N))) {
                        for (int j = 0; j < N; j++) x[j] = make_double2(sum[j].x / sample, sum[j].y / sample);
                        rec.t = 1.0;
                        // the relative residual of the estimate decides whether it counts
                        for (int j = 0; j < N; j++) SL(xe, j) = x[j];
                        evaluate<N, double2, true>(C0, C1, tb, 1.0, false, true, xe, R, J, P, S, bt);
                        double rr = 0.0;
                        for (int i = 0; i < N; i++) {
                            const double r = abs1(SL(R, i)) / (1.0 + SL(S, i).x);
                            if (!(r <= rr)) rr = r;
                        }
                        rec.relres = rr;
                        cycle = (rr <= EG_RES) ? sample / EG_SAMPLES : -1;
                    }
                }
            }
            if (cycle < 0) cycle = 0;
        }
        rec.stop = stop;
        rec.norm_x = norm_n(x, N);
        for (int j = 0; j < N; j++) L.x_out[(int64_t)j * np + q] = x[j];
        L.stats[q] = rec;
        cycle_out[q] = cycle;
    }
}

template <int N>
static cudaError_t launch_endgame_n(const TrackLaunch &L, int32_t *cycle_out, int block_threads, int max_blocks,
                                    cudaStream_t s)
{
    const size_t tb = table_smem_bytes(L.tab);
    int bt = track_block_threads(N, tb, block_threads, true, false);
    if (bt > 128) bt = 128;
    if (bt == 0) return cudaErrorInvalidConfiguration;
    const size_t smem = tb + (size_t)bt * thread_smem_bytes(N, true, false);
    cudaError_t e = cudaFuncSetAttribute(endgame_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, endgame_kernel<N>, bt, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int64_t want = (L.n_paths + bt - 1) / bt;
    int64_t grid = (int64_t)g_num_sms * per_sm;
    if (max_blocks > 0 && grid > max_blocks) grid = max_blocks;
    if (grid > want) grid = want;
    if (grid < 1) grid = 1;
    endgame_kernel<N><<<(unsigned)grid, bt, smem, s>>>(L, tb, cycle_out);
    return cudaGetLastError();
}

cudaError_t launch_endgame(const TrackLaunch &L, int32_t *cycle_out, int block_threads, int max_blocks, cudaStream_t s)
{
    device_limits();
    if (L.n_paths <= 0) return cudaSuccess;
#define PHC_CALL_EG(NN) launch_endgame_n<NN>(L, cycle_out, block_threads, max_blocks, s)
    PHC_DISPATCH_N(L.tab.n, PHC_CALL_EG)
#undef PHC_CALL_EG
}

}  // namespace phc
