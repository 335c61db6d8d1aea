// track_qd.cu -- path tracking in complex quad double arithmetic.
//
// Section 5 and Table 2 run the paper's whole solver in quad double as well
// as double double ("quality up").  This kernel tracks total-degree paths with
// the readings of track_kernel -- RK4 predictor, Newton corrector, the same
// step control, tolerances, stall and divergence rules -- with the point x,
// the Runge-Kutta stages, H, H_x, H_t, the LU and the solves in complex quad
// double (qd.cuh); t, the step sizes and the norms (from the leading parts)
// stay double.  The end Newton at t = 1 stops at ||dx|| <= 1e-58 (1 + ||x||).
// The classification pass (classify_kernel) works on the leading parts, as
// for a double precision endpoint.
//
// One thread per path.  A complex quad double is 64 bytes, so a thread's
// Jacobian alone takes N^2 x 64 bytes: the thread's arrays live in its local
// memory (L1, then L2) rather than in shared memory, which holds the term
// table.  Every quad double operation costs tens to hundreds of FP64
// instructions per byte it touches, so the kernel is bound by the FP64 pipe.
#include "qd.cuh"
#include "track_impl.cuh"

namespace phc {

#define END_TOL_QD 1e-58

__device__ __forceinline__ cqd cqd_of(double2 c) { return cqd_from(c.x, c.y); }

// J = H_x (row-major N x N) and R = H_t (dt) or H (!dt) at (X, t) for the
// homotopy sum_q (c0_q + t c1_q) x^{a_q}: per term the common factor
// cf = prod x_{v_j}^{a_j - 1}, prefix products P_j = c(t) cf prod_{i<j} x_{v_i}
// and suffix products (Speelpenning), as add_term does in double precision.
template <int N>
__device__ void evaluate_qd(const SmTab &tb, const double2 *C0, const double2 *C1, double t, bool dt, const cqd *X,
                            cqd *R, cqd *J)
{
    const cqd zero = cqd_from(0.0, 0.0), one = cqd_from(1.0, 0.0);
    for (int i = 0; i < N; i++) R[i] = zero;
    for (int i = 0; i < N * N; i++) J[i] = zero;
    cqd pre[N];
    for (int q = 0; q < tb.n_terms; q++) {
        const TermRec r = tb.terms[q];
        const cqd c1 = cqd_of(C1[q]);
        const cqd ct = cqd_add(cqd_of(C0[q]), cqd_scale(t, c1));
        const cqd cr = dt ? c1 : ct;
        if (r.k == 0) {
            R[r.eq] = cqd_add(R[r.eq], cr);
            continue;
        }
        const uint8_t *v = tb.vars + r.off;
        const uint8_t *e = tb.exps + r.off;
        const int k = r.k;
        cqd cf = one;
        if (r.flags & TERM_POWERS) {
            for (int j = 0; j < k; j++) {
                if (e[j] > 1) {
                    const cqd xv = X[v[j]];
                    cqd pw = xv;
                    for (int m = 2; m < e[j]; m++) pw = cqd_mul(pw, xv);
                    cf = cqd_mul(cf, pw);
                }
            }
            pre[0] = cqd_mul(ct, cf);
        } else {
            pre[0] = ct;
        }
        for (int j = 1; j < k; j++) pre[j] = cqd_mul(pre[j - 1], X[v[j - 1]]);
        cqd suf = X[v[k - 1]];
        const int row = r.eq * N;
        J[row + v[k - 1]] = cqd_add(J[row + v[k - 1]], cqd_scale((double)e[k - 1], pre[k - 1]));
        for (int j = k - 2; j >= 0; j--) {
            J[row + v[j]] = cqd_add(J[row + v[j]], cqd_mul(cqd_scale((double)e[j], pre[j]), suf));
            suf = cqd_mul(suf, X[v[j]]);
        }
        R[r.eq] = cqd_add(R[r.eq], cqd_mul(cr, cqd_mul(cf, suf)));
    }
}

// Solves J y = R in place (R := y) by LU with partial pivoting by the largest
// |.|_1 of the leading parts (the first row on ties), J overwritten.  Returns
// false on a zero pivot.
template <int N>
__device__ bool lu_solve_qd(cqd *J, cqd *R)
{
    for (int k = 0; k < N; k++) {
        int p = k;
        double best = cqd_abs1(J[k * N + k]);
        for (int i = k + 1; i < N; i++) {
            const double a = cqd_abs1(J[i * N + k]);
            if (a > best) {
                best = a;
                p = i;
            }
        }
        if (!(best > 0.0)) return false;
        if (p != k) {
            for (int j = 0; j < N; j++) {
                const cqd a = J[k * N + j];
                J[k * N + j] = J[p * N + j];
                J[p * N + j] = a;
            }
            const cqd a = R[k];
            R[k] = R[p];
            R[p] = a;
        }
        const cqd piv = J[k * N + k];
        for (int i = k + 1; i < N; i++) {
            const cqd l = cqd_div(J[i * N + k], piv);
            for (int j = k + 1; j < N; j++) J[i * N + j] = cqd_sub(J[i * N + j], cqd_mul(l, J[k * N + j]));
            R[i] = cqd_sub(R[i], cqd_mul(l, R[k]));
        }
    }
    for (int i = N - 1; i >= 0; i--) {
        cqd s = R[i];
        for (int j = i + 1; j < N; j++) s = cqd_sub(s, cqd_mul(J[i * N + j], R[j]));
        R[i] = cqd_div(s, J[i * N + i]);
    }
    return true;
}

template <int N>
__global__ void __launch_bounds__(128) track_qd_kernel(const TrackLaunch L, size_t table_bytes)
{
    extern __shared__ __align__(16) char smem[];
    const SmTab tb = stage_table(L.tab, smem);
    const phc_opts &o = L.o;
    const int64_t np = L.n_paths;
    cqd x0[N], acc[N], xe[N], R[N], J[N * N];
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
            const double2 z = L.roots[L.root_off[i] + k];
            x0[i] = cqd_from(z.x, z.y);
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
            bool ok = true;
            // predictor: RK4, k_s = -J^{-1} H_t at the stage points
            for (int j = 0; j < N; j++) xe[j] = x0[j];
            for (int stage = 0; stage < 4 && ok; stage++) {
                const double ts = stage == 0 ? t : stage < 3 ? t + 0.5 * he : t1;
                evaluate_qd<N>(tb, C0, C1, ts, true, xe, R, J);
                n_solve++;
                ok = lu_solve_qd<N>(J, R);
                if (!ok) break;
                for (int j = 0; j < N; j++) {
                    const cqd kj = cqd_neg(R[j]);
                    acc[j] = stage == 0 ? kj : cqd_add(acc[j], stage == 3 ? kj : cqd_scale(2.0, kj));
                    if (stage < 2) xe[j] = cqd_add(x0[j], cqd_scale(0.5 * he, kj));
                    else if (stage == 2) xe[j] = cqd_add(x0[j], cqd_scale(he, kj));
                }
            }
            if (ok)
                for (int j = 0; j < N; j++) xe[j] = cqd_add(x0[j], cqd_scale(he / 6.0, acc[j]));
            // corrector: Newton at t1
            bool conv = false;
            double prev = 0.0;
            for (int it = 0; ok && it < o.max_corr_iters; it++) {
                evaluate_qd<N>(tb, C0, C1, t1, false, xe, R, J);
                n_solve++;
                n_newt++;
                if (!lu_solve_qd<N>(J, R)) break;
                double d = 0.0, nx = 0.0;
                bool fin = true;
                for (int j = 0; j < N; j++) {
                    xe[j] = cqd_sub(xe[j], R[j]);
                    const double a = cqd_absinf(R[j]);
                    if (!(a <= d)) d = a;
                    const double b = cqd_absinf(xe[j]);
                    if (!(b <= nx)) nx = b;
                    fin = fin && cqd_finite(xe[j]);
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
                    x0[j] = xe[j];
                    const double a = cqd_absinf(x0[j]);
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
            for (int j = 0; j < N; j++) xe[j] = x0[j];
            for (int it = 0; it < o.end_iters; it++) {
                evaluate_qd<N>(tb, C0, C1, 1.0, false, xe, R, J);
                n_solve++;
                n_newt++;
                if (!lu_solve_qd<N>(J, R)) break;
                double d = 0.0, nx = 0.0;
                bool fin = true;
                for (int j = 0; j < N; j++) {
                    xe[j] = cqd_sub(xe[j], R[j]);
                    x0[j] = xe[j];
                    const double a = cqd_absinf(R[j]);
                    if (!(a <= d)) d = a;
                    const double b = cqd_absinf(xe[j]);
                    if (!(b <= nx)) nx = b;
                    fin = fin && cqd_finite(xe[j]);
                }
                if (!(d == d) || !fin) break;
                if (d <= END_TOL_QD * (1.0 + nx)) break;
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
        // parts 0..3 of every coordinate: x_out + part * N * np (SoA [4][N][np])
        for (int j = 0; j < N; j++) {
            const int64_t at = (int64_t)j * np + q, part = (int64_t)N * np;
            L.x_out[at] = make_double2(x0[j].re.x0, x0[j].im.x0);
            L.x_out[at + part] = make_double2(x0[j].re.x1, x0[j].im.x1);
            L.x_out[at + 2 * part] = make_double2(x0[j].re.x2, x0[j].im.x2);
            L.x_out[at + 3 * part] = make_double2(x0[j].re.x3, x0[j].im.x3);
        }
        L.stats[q] = rec;
    }
}

template <int N>
static cudaError_t launch_track_qd_n(const TrackLaunch &L, int block_threads, int max_blocks, cudaStream_t s)
{
    const size_t tb = table_smem_bytes(L.tab);
    if (tb > (size_t)g_smem_optin) return cudaErrorInvalidConfiguration;
    int bt = 128;
    if (block_threads > 0 && block_threads < bt) bt = block_threads < 32 ? 32 : (block_threads / 32) * 32;
    cudaError_t e = cudaFuncSetAttribute(track_qd_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tb);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, track_qd_kernel<N>, bt, tb);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int64_t want = (L.n_paths + bt - 1) / bt;
    int64_t grid = (int64_t)g_num_sms * per_sm;
    if (max_blocks > 0 && grid > max_blocks) grid = max_blocks;
    if (grid > want) grid = want;
    if (grid < 1) grid = 1;
    track_qd_kernel<N><<<(unsigned)grid, bt, tb, s>>>(L, tb);
    return cudaGetLastError();
}

cudaError_t launch_track_qd(const TrackLaunch &L, int block_threads, int max_blocks, cudaStream_t s)
{
    device_limits();
    if (L.n_paths <= 0) return cudaSuccess;
#define PHC_CALL_QD(NN) launch_track_qd_n<NN>(L, block_threads, max_blocks, s)
    PHC_DISPATCH_N(L.tab.n, PHC_CALL_QD)
#undef PHC_CALL_QD
}

}  // namespace phc
