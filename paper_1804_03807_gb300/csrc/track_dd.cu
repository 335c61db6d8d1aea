// track_dd.cu -- path tracking in complex double double arithmetic.
//
// Section 5 and Table 2 run the paper's whole solver in double double
// arithmetic ("quality up").  This kernel tracks total-degree paths with the
// readings of track_kernel -- RK4 predictor, Newton corrector, the same step
// control, tolerances, stall and divergence rules -- but the point x, the
// Runge-Kutta stages, H, H_x, H_t, the LU and the solves are complex double
// double; t, the step sizes and the norms (taken from the double parts) stay
// double.  The end Newton at t = 1 stops at ||dx|| <= 1e-26 (1 + ||x||).  The
// classification pass (classify_kernel) then works on the double parts, as for
// a double precision endpoint.
//
// One thread per path, as in track_kernel; a complex double double takes two
// shared-memory slots of the thread (the double parts (re.hi, im.hi), then
// (re.lo, im.lo)), element-major and lane-fastest.  A unit costs about 15
// times the double precision unit, so there is no tail hand-off and no
// compaction: this tracker is for the paths that need the accuracy.
#include "dd.cuh"
#include "track_impl.cuh"

namespace phc {

__device__ __forceinline__ cdd ldd(const double2 *a, int i, int bt)
{
    const double2 h = a[(2 * i) * bt], l = a[(2 * i + 1) * bt];
    return {{h.x, l.x}, {h.y, l.y}};
}
__device__ __forceinline__ void sdd(double2 *a, int i, int bt, cdd v)
{
    a[(2 * i) * bt] = make_double2(v.re.hi, v.im.hi);
    a[(2 * i + 1) * bt] = make_double2(v.re.lo, v.im.lo);
}
__device__ __forceinline__ double cdd_norm_hi(cdd a) { return cdd_absinf(a); }
__device__ __forceinline__ bool cdd_finite(cdd a)
{
    return isfinite(a.re.hi) && isfinite(a.im.hi) && isfinite(a.re.lo) && isfinite(a.im.lo);
}

// J = H_x (row-major N x N) and R = H_t (dt) or H (!dt) at (X, t) for the
// homotopy sum_q (c0_q + t c1_q) x^{a_q}: per term the common factor
// cf = prod x_{v_j}^{a_j - 1}, prefix products P_j = c(t) cf prod_{i<j} x_{v_i}
// (in local memory) and suffix products (Speelpenning), as add_term does in
// double precision.
template <int N>
__device__ void evaluate_dd(const SmTab &tb, const double2 *C0, const double2 *C1, double t, bool dt,
                            const double2 *X, double2 *R, double2 *J, int bt)
{
    const cdd zero = {{0.0, 0.0}, {0.0, 0.0}};
    const cdd one = {{1.0, 0.0}, {0.0, 0.0}};
#pragma unroll
    for (int i = 0; i < N; i++) sdd(R, i, bt, zero);
    for (int i = 0; i < N * N; i++) sdd(J, i, bt, zero);
    const cdd tt = {{t, 0.0}, {0.0, 0.0}};
    cdd pre[N];
    for (int q = 0; q < tb.n_terms; q++) {
        const TermRec r = tb.terms[q];
        const cdd c0 = cdd_from(C0[q]), c1 = cdd_from(C1[q]);
        const cdd ct = cdd_add(c0, cdd_mul(tt, c1));
        const cdd cr = dt ? c1 : ct;
        double2 *Rrow = R, *Jrow = J;
        if (r.k == 0) {
            sdd(Rrow, r.eq, bt, cdd_add(ldd(Rrow, r.eq, bt), cr));
            continue;
        }
        const uint8_t *v = tb.vars + r.off;
        const uint8_t *e = tb.exps + r.off;
        const int k = r.k;
        cdd cf = one;
        if (r.flags & TERM_POWERS) {
            for (int j = 0; j < k; j++) {
                if (e[j] > 1) {
                    const cdd xv = ldd(X, v[j], bt);
                    cdd pw = xv;
                    for (int m = 2; m < e[j]; m++) pw = cdd_mul(pw, xv);
                    cf = cdd_mul(cf, pw);
                }
            }
            pre[0] = cdd_mul(ct, cf);
        } else {
            pre[0] = ct;
        }
        for (int j = 1; j < k; j++) pre[j] = cdd_mul(pre[j - 1], ldd(X, v[j - 1], bt));
        cdd suf = ldd(X, v[k - 1], bt);
        const int row = r.eq * N;
        sdd(Jrow, row + v[k - 1], bt, cdd_add(ldd(Jrow, row + v[k - 1], bt), cdd_scale((double)e[k - 1], pre[k - 1])));
        for (int j = k - 2; j >= 0; j--) {
            const cdd d = cdd_mul(cdd_scale((double)e[j], pre[j]), suf);
            sdd(Jrow, row + v[j], bt, cdd_add(ldd(Jrow, row + v[j], bt), d));
            suf = cdd_mul(suf, ldd(X, v[j], bt));
        }
        const cdd mono = cdd_mul(cf, suf);
        sdd(Rrow, r.eq, bt, cdd_add(ldd(Rrow, r.eq, bt), cdd_mul(cr, mono)));
    }
}

// Solves J y = R in place (R := y) by LU with partial pivoting by the
// largest |.|_1 of the double parts (the first row on ties), J overwritten.
// Returns false on a zero pivot.
template <int N>
__device__ bool lu_solve_dd(double2 *J, double2 *R, int bt)
{
    for (int k = 0; k < N; k++) {
        int p = k;
        double best = cdd_abs1(ldd(J, k * N + k, bt));
        for (int i = k + 1; i < N; i++) {
            const double a = cdd_abs1(ldd(J, i * N + k, bt));
            if (a > best) {
                best = a;
                p = i;
            }
        }
        if (!(best > 0.0)) return false;
        if (p != k) {
            for (int j = 0; j < N; j++) {
                const cdd a = ldd(J, k * N + j, bt), c = ldd(J, p * N + j, bt);
                sdd(J, k * N + j, bt, c);
                sdd(J, p * N + j, bt, a);
            }
            const cdd a = ldd(R, k, bt), c = ldd(R, p, bt);
            sdd(R, k, bt, c);
            sdd(R, p, bt, a);
        }
        const cdd piv = ldd(J, k * N + k, bt);
        for (int i = k + 1; i < N; i++) {
            const cdd l = cdd_div(ldd(J, i * N + k, bt), piv);
            for (int j = k + 1; j < N; j++)
                sdd(J, i * N + j, bt, cdd_sub(ldd(J, i * N + j, bt), cdd_mul(l, ldd(J, k * N + j, bt))));
            sdd(R, i, bt, cdd_sub(ldd(R, i, bt), cdd_mul(l, ldd(R, k, bt))));
        }
    }
    for (int i = N - 1; i >= 0; i--) {
        cdd s = ldd(R, i, bt);
        for (int j = i + 1; j < N; j++) s = cdd_sub(s, cdd_mul(ldd(J, i * N + j, bt), ldd(R, j, bt)));
        sdd(R, i, bt, cdd_div(s, ldd(J, i * N + i, bt)));
    }
    return true;
}

#define END_TOL_DD 1e-26

template <int N>
__global__ void __launch_bounds__(128) track_dd_kernel(const TrackLaunch L, size_t table_bytes)
{
    extern __shared__ __align__(16) char smem[];
    const SmTab tb = stage_table(L.tab, smem);
    const int bt = blockDim.x;
    double2 *xe = reinterpret_cast<double2 *>(smem + table_bytes) + threadIdx.x;
    double2 *R = xe + 2 * N * bt;
    double2 *J = R + 2 * N * bt;
    const phc_opts &o = L.o;
    const int64_t np = L.n_paths;
    cdd x0[N], acc[N], sol[N];
    for (;;) {
        const unsigned long long c = atomicAdd(L.qhead, 1ull);
        if (c >= (unsigned long long)np) break;
        const int64_t q = (int64_t)c;
        const int64_t gid = L.first + q;
        const int sys = (int)(gid / L.paths_per_system);
        int64_t pid = gid - (int64_t)sys * L.paths_per_system;
        for (int i = 0; i < N; i++) {
            const int d = L.deg[i];
            const int k = (int)(pid % d);
            pid /= d;
            x0[i] = cdd_from(L.roots[L.root_off[i] + k]);
        }
        const double2 *C0 = tb.c0 + (size_t)sys * tb.n_terms, *C1 = tb.c1 + (size_t)sys * tb.n_terms;
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
            const cdd hh = {{0.5 * he, 0.0}, {0.0, 0.0}}, hf = {{he, 0.0}, {0.0, 0.0}};
            const cdd h6 = {{he / 6.0, 0.0}, {0.0, 0.0}}, two = {{2.0, 0.0}, {0.0, 0.0}};
            bool ok = true;
            // predictor: RK4, k_s = -J^{-1} H_t at the stage points
            for (int j = 0; j < N; j++) sdd(xe, j, bt, x0[j]);
            for (int stage = 0; stage < 4 && ok; stage++) {
                const double ts = stage == 0 ? t : stage < 3 ? t + 0.5 * he : t1;
                evaluate_dd<N>(tb, C0, C1, ts, true, xe, R, J, bt);
                n_solve++;
                ok = lu_solve_dd<N>(J, R, bt);
                if (!ok) break;
                for (int j = 0; j < N; j++) {
                    const cdd kj = cdd_neg(ldd(R, j, bt));
                    acc[j] = stage == 0 ? kj : cdd_add(acc[j], stage == 3 ? kj : cdd_mul(two, kj));
                    if (stage < 2) sdd(xe, j, bt, cdd_add(x0[j], cdd_mul(hh, kj)));
                    else if (stage == 2) sdd(xe, j, bt, cdd_add(x0[j], cdd_mul(hf, kj)));
                }
            }
            if (ok)
                for (int j = 0; j < N; j++) sdd(xe, j, bt, cdd_add(x0[j], cdd_mul(h6, acc[j])));
            // corrector: Newton at t1
            bool conv = false;
            double prev = 0.0;
            for (int it = 0; ok && it < o.max_corr_iters; it++) {
                evaluate_dd<N>(tb, C0, C1, t1, false, xe, R, J, bt);
                n_solve++;
                n_newt++;
                if (!lu_solve_dd<N>(J, R, bt)) break;
                double d = 0.0, nx = 0.0;
                bool fin = true;
                for (int j = 0; j < N; j++) {
                    const cdd dj = ldd(R, j, bt);
                    const cdd xj = cdd_sub(ldd(xe, j, bt), dj);
                    sdd(xe, j, bt, xj);
                    const double a = cdd_norm_hi(dj);
                    if (!(a <= d)) d = a;
                    const double b = cdd_norm_hi(xj);
                    if (!(b <= nx)) nx = b;
                    fin = fin && cdd_finite(xj);
                }
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
                for (int j = 0; j < N; j++) {
                    x0[j] = ldd(xe, j, bt);
                    const double a = cdd_norm_hi(x0[j]);
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
            for (int j = 0; j < N; j++) sdd(xe, j, bt, x0[j]);
            for (int it = 0; it < o.end_iters; it++) {
                evaluate_dd<N>(tb, C0, C1, 1.0, false, xe, R, J, bt);
                n_solve++;
                n_newt++;
                if (!lu_solve_dd<N>(J, R, bt)) break;
                double d = 0.0, nx = 0.0;
                bool fin = true;
                for (int j = 0; j < N; j++) {
                    const cdd dj = ldd(R, j, bt);
                    const cdd xj = cdd_sub(ldd(xe, j, bt), dj);
                    sdd(xe, j, bt, xj);
                    x0[j] = xj;
                    const double a = cdd_norm_hi(dj);
                    if (!(a <= d)) d = a;
                    const double b = cdd_norm_hi(xj);
                    if (!(b <= nx)) nx = b;
                    fin = fin && cdd_finite(xj);
                }
                if (!(d == d) || !fin) break;
                if (d <= END_TOL_DD * (1.0 + nx)) break;
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
        rec.system = sys;
        for (int j = 0; j < N; j++) {
            L.x_out[(int64_t)j * np + q] = make_double2(x0[j].re.hi, x0[j].im.hi);
            L.x_out2[(int64_t)j * np + q] = make_double2(x0[j].re.lo, x0[j].im.lo);
        }
        L.stats[q] = rec;
    }
}

// Per-thread shared memory of the double double tracker: xe, R (N each) and
// J (N^2), two slots per complex double double.
static size_t dd_thread_bytes(int n) { return (size_t)(n * n + 2 * n) * 2 * sizeof(double2); }

template <int N>
static cudaError_t launch_track_dd_n(const TrackLaunch &L, int block_threads, int max_blocks, cudaStream_t s)
{
    const size_t tb = table_smem_bytes(L.tab);
    long fit = ((long)g_smem_optin - (long)tb) / (long)dd_thread_bytes(N);
    int bt = (int)((fit / 32) * 32);
    if (bt > 128) bt = 128;
    if (block_threads > 0 && block_threads < bt) bt = (block_threads / 32) * 32;
    if (bt < 32) return cudaErrorInvalidConfiguration;
    const size_t smem = tb + (size_t)bt * dd_thread_bytes(N);
    cudaError_t e = cudaFuncSetAttribute(track_dd_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, track_dd_kernel<N>, bt, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int64_t want = (L.n_paths + bt - 1) / bt;
    int64_t grid = (int64_t)g_num_sms * per_sm;
    if (max_blocks > 0 && grid > max_blocks) grid = max_blocks;
    if (grid > want) grid = want;
    if (grid < 1) grid = 1;
    track_dd_kernel<N><<<(unsigned)grid, bt, smem, s>>>(L, tb);
    return cudaGetLastError();
}

cudaError_t launch_track_dd(const TrackLaunch &L, int block_threads, int max_blocks, cudaStream_t s)
{
    device_limits();
    if (L.n_paths <= 0) return cudaSuccess;
#define PHC_CALL_DD(NN) launch_track_dd_n<NN>(L, block_threads, max_blocks, s)
    PHC_DISPATCH_N(L.tab.n, PHC_CALL_DD)
#undef PHC_CALL_DD
}

}  // namespace phc
