// track_tail.cu -- the row-parallel tail kernel.
//
// When most lanes of a tracking launch have run out of paths, the remaining
// paths leave the one-thread-per-path kernel at the start of a step (see the
// hand-off in track_impl.cuh) and continue here with G lanes per path: lane
// r owns equation r -- its terms in the evaluation, row r of the Jacobian in
// the LU and in the triangular solves.  A long path then no longer runs at the
// speed of one thread sharing an FP64 pipe with a partly empty warp.
//
// Every value is computed by exactly the operations, in exactly the order,
// of the one-thread kernel (terms of a row in table order, one column
// elimination at a time, forward substitution over ascending and back
// substitution over descending columns), and the scalars of the step logic
// are reduced with exact operations (max, and), so a path ends with the same
// bits whichever kernel finishes it.
#include "track_impl.cuh"

namespace phc {

template <int G>
__device__ __forceinline__ double gmax(double v, unsigned mask)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        const double w = __shfl_xor_sync(mask, v, o, G);
        v = (w > v) ? w : v;
    }
    return v;
}

template <int N, int G>
__global__ void __launch_bounds__(128) tail_kernel(const TrackLaunch L, size_t table_bytes)
{
    extern __shared__ __align__(16) char smem[];
    const SmTab tb = stage_table(L.tab, smem);
    // The terms of equation i are tb.terms[rs[i] .. rs[i + 1]) (tables are
    // grouped by equation in ascending order); mt = most terms of one row.
    __shared__ int rs[PHC_MAX_VARS + 1], mt;
    if (threadIdx.x == 0) {
        int q = 0, m = 0;
        for (int i = 0; i < N; i++) {
            rs[i] = q;
            while (q < tb.n_terms && tb.terms[q].eq == i) q++;
            m = (q - rs[i] > m) ? q - rs[i] : m;
        }
        rs[N] = q;
        mt = m;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int r = lane % G;  // the equation / row this lane owns (r < N)
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane - r));
    const int group = threadIdx.x / G;
    constexpr int SLOTS = 2 * N + N * N + G * N;
    double2 *base = reinterpret_cast<double2 *>(smem + table_bytes) + (size_t)group * SLOTS;
    double2 *xe = base;          // [N]
    double2 *R = base + N;       // [N]
    double2 *J = base + 2 * N;   // [N][N]
    double2 *P = base + 2 * N + N * N + r * N;  // this lane's prefix products
    const phc_opts &o = L.o;
    const int64_t np = L.n_paths;
    const bool own = r < N;
    const unsigned long long n_hand = *reinterpret_cast<volatile const unsigned long long *>(L.handoff_n);

    for (;;) {
        unsigned long long slot = 0;
        if (r == 0) slot = atomicAdd(L.tail_q, 1ull);
        slot = __shfl_sync(gmask, slot, 0, G);
        if (slot >= n_hand) break;
        const Handoff &hd = L.handoff[slot];
        double t = hd.t, h = hd.h, next_s = hd.next_s;
        double r0 = hd.r0, r1 = hd.r1, r2 = hd.r2, r3 = hd.r3, r4 = hd.r4;
        const int64_t q = hd.q;
        const int sys = hd.sys;
        int streak = hd.streak, steps = hd.steps, since_ck = hd.since_ck, nck = hd.nck;
        int n_acc = hd.n_acc, n_rej = hd.n_rej, n_newt = hd.n_newt, n_solve = hd.n_solve;
        const int n_f32 = hd.n_f32;
        double2 x0r = own ? hd.x0[r] : make_double2(0.0, 0.0);
        double2 accr = make_double2(0.0, 0.0), solr = make_double2(0.0, 0.0);
        double he = 0.0, t1 = 0.0, te = 0.0, prev = 0.0;
        int phase = 0, it = 0;
        const double2 *C0 = tb.c0 + (size_t)sys * tb.n_terms, *C1 = tb.c1 + (size_t)sys * tb.n_terms;

        auto begin_step = [&]() {
            he = h;
            t1 = t + he;
            if (he >= 1.0 - t) {
                he = 1.0 - t;
                t1 = 1.0;
            }
            if (own) xe[r] = x0r;
            accr = make_double2(0.0, 0.0);
            te = t;
            phase = 0;
        };
        begin_step();
        int stop = -1;
        for (;;) {
            __syncwarp(gmask);
            // ---------------------------------------------- evaluate row r (as evaluate<N, double2>, same add_term)
            const bool dt = phase < 4;
            if (own) {
                const double2 zero = make_double2(0.0, 0.0);
                R[r] = zero;
#pragma unroll
                for (int j = 0; j < N; j++) J[r * N + j] = zero;
                // the terms of equation r, in table order; the lanes of a
                // group step through their rows together (term i of every row)
                const int q0 = rs[r], q1 = rs[r + 1];
                for (int i = 0; i < mt; i++) {
                    const int qq = q0 + i;
                    if (qq >= q1) continue;
                    const TermRec rec = tb.terms[qq];
                    const double2 c0 = C0[qq], c1 = C1[qq];
                    const double2 ct = make_double2(fma(te, c1.x, c0.x), fma(te, c1.y, c0.y));
                    const double2 cr = dt ? c1 : ct;
                    if (rec.k == 0) {
                        R[r] = cadd(R[r], cr);
                        continue;
                    }
                    add_term<double2>(rec, tb.vars + rec.off, tb.exps + rec.off, ct, cr, true, xe, J + r * N, R + r,
                                      P, 1);
                }
            }
            __syncwarp(gmask);
            // ---------------------------------------------- LU (as lu_factor<N, double2>)
            bool ok = true;
            int perm[N];
#pragma unroll
            for (int k = 0; k < N; k++) {
                const double vk = abs1(J[k * N + k]);
                // candidates: rows i > k with a larger |.|_1 (the first on ties)
                double bv = (own && r > k) ? abs1(J[r * N + k]) : -1.0;
                if (!(bv == bv)) bv = -1.0;
                int bi = (own && r > k) ? r : N;
#pragma unroll
                for (int off = G / 2; off > 0; off >>= 1) {
                    const double ov = __shfl_xor_sync(gmask, bv, off, G);
                    const int oi = __shfl_xor_sync(gmask, bi, off, G);
                    if (ov > bv || (ov == bv && oi < bi)) {
                        bv = ov;
                        bi = oi;
                    }
                }
                int p = k;
                double best = vk;
                if (bi < N && bv > best) {
                    best = bv;
                    p = bi;
                }
                perm[k] = p;
                if (!(best > 0.0)) {
                    ok = false;
                    break;
                }
                __syncwarp(gmask);  // every lane has read column k before row k changes
                if (own && p != k) {
                    const double2 a = J[k * N + r], c = J[p * N + r];
                    J[k * N + r] = c;
                    J[p * N + r] = a;
                }
                __syncwarp(gmask);
                const double2 inv = recip(J[k * N + k]);
                __syncwarp(gmask);
                if (r == k) J[k * N + k] = inv;
                if (own && r > k) {
                    const double2 l = cmul(J[r * N + k], inv);
                    J[r * N + k] = l;
#pragma unroll
                    for (int j = k + 1; j < N; j++) J[r * N + j] = cfms(J[r * N + j], l, J[k * N + j]);
                }
                __syncwarp(gmask);
            }
            // ---------------------------------------------- solve (as lu_solve<N, double2>)
            if (ok) {
                if (r == 0) {
#pragma unroll
                    for (int k = 0; k < N; k++) {
                        const int p = perm[k];
                        const double2 a = R[k], c = R[p];
                        R[k] = c;
                        R[p] = a;
                    }
                }
                __syncwarp(gmask);
#pragma unroll
                for (int k = 0; k < N - 1; k++) {
                    if (own && r > k) R[r] = cfms(R[r], J[r * N + k], R[k]);
                    __syncwarp(gmask);
                }
#pragma unroll
                for (int k = N - 1; k >= 0; k--) {
                    if (r == k) R[k] = cmul(R[k], J[k * N + k]);
                    __syncwarp(gmask);
                    if (own && r < k) R[r] = cfms(R[r], J[r * N + k], R[k]);
                    __syncwarp(gmask);
                }
            }
            solr = (own && ok) ? R[r] : make_double2(0.0, 0.0);
            n_solve++;
            __syncwarp(gmask);

            // ---------------------------------------------- what the unit was for
            enum { ACT_NONE = 0, ACT_ACCEPT, ACT_REJECT };
            int act = ACT_NONE;
            if (phase < 4) {
                const bool fin = __all_sync(gmask, !own || (ok && finite2(solr)));
                if (!ok || !fin) {
                    act = ACT_REJECT;
                } else {
                    const double wacc = (phase == 0 || phase == 3) ? 1.0 : 2.0;
                    const double hs = (phase < 2) ? 0.5 * he : he;
                    if (own) {
                        const double2 kj = make_double2(-solr.x, -solr.y);
                        accr = (phase == 0) ? kj : caxpy(accr, wacc, kj);
                        xe[r] = (phase < 3) ? caxpy(x0r, hs, kj) : caxpy(x0r, he / 6.0, accr);
                    }
                    te = (phase < 2) ? t + 0.5 * he : t1;
                    if (phase == 3) {
                        it = 0;
                        prev = 0.0;
                    }
                    phase++;
                }
            } else {
                n_newt++;
                double a = 0.0, c = 0.0;
                bool fl = true;
                if (ok && own) {
                    const double2 xj = make_double2(xe[r].x - solr.x, xe[r].y - solr.y);
                    xe[r] = xj;
                    if (phase == 5) x0r = xj;
                    a = absinf(solr);
                    c = absinf(xj);
                    fl = finite2(xj);
                }
                const bool fin = __all_sync(gmask, fl);
                const double d = fin ? gmax<G>(a, gmask) : NAN;
                const double nx = fin ? gmax<G>(c, gmask) : NAN;
                if (phase == 4) {
                    if (!ok || !(d == d) || !fin) act = ACT_REJECT;
                    else if (d <= o.corr_tol * (1.0 + nx)) act = ACT_ACCEPT;
                    else if (it > 0 && d > o.corr_contract * prev) act = ACT_REJECT;
                    else {
                        prev = d;
                        if (++it >= o.max_corr_iters) act = ACT_REJECT;
                    }
                } else {
                    if (!ok) stop = PHC_STOP_REACHED;
                    else if (!(d == d) || !fin) stop = fin ? PHC_STOP_REACHED : PHC_STOP_NONFINITE;
                    else if (d <= o.end_tol * (1.0 + nx) || ++it >= o.end_iters) stop = PHC_STOP_REACHED;
                }
            }
            __syncwarp(gmask);

            // ---------------------------------------------- step control
            if (act == ACT_ACCEPT) {
                t = t1;
                if (own) x0r = xe[r];
                const double nx = gmax<G>(own ? absinf(x0r) : 0.0, gmask);
                n_acc++;
                steps++;
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
                } else {
                    if (++streak >= o.expand_after) {
                        streak = 0;
                        h = h * o.expand;
                        if (h > o.h_max) h = o.h_max;
                    }
                    if (steps >= o.max_steps) stop = PHC_STOP_BUDGET;
                    else if (++since_ck >= o.max_steps_decade && t < 1.0) stop = PHC_STOP_BUDGET;
                    else if (t >= 1.0) {
                        phase = 5;
                        it = 0;
                        te = 1.0;
                    } else {
                        begin_step();
                    }
                }
            } else if (act == ACT_REJECT) {
                n_rej++;
                steps++;
                streak = 0;
                h = he * o.shrink;
                if (h < o.h_min) stop = PHC_STOP_STEP_MIN;
                if (stop < 0 && steps >= o.max_steps) stop = PHC_STOP_BUDGET;
                if (stop < 0 && ++since_ck >= o.max_steps_decade) stop = PHC_STOP_BUDGET;
                if (stop < 0) begin_step();
            }
            if (stop >= 0) break;
        }

        // ---------------------------------------------- the path ends
        if (own) L.x_out[(int64_t)r * np + q] = x0r;
        if (r == 0) {
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
            rec.n_fp32 = n_f32;
            rec.grew = grew;
            rec.system = sys;
            L.stats[q] = rec;
        }
        __syncwarp(gmask);
    }
}

template <int N, int G>
static cudaError_t launch_tail_n(const TrackLaunch &L_in, int max_blocks, cudaStream_t s)
{
    TrackLaunch L = L_in;
    L.tab.coef_smem = 1;  // this kernel's shared memory is small
    const size_t tb = table_smem_bytes(L.tab);
    const int bt = 128;
    const size_t smem = tb + (size_t)(bt / G) * (2 * N + N * N + G * N) * sizeof(double2);
    cudaError_t e = cudaFuncSetAttribute(tail_kernel<N, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tail_kernel<N, G>, bt, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int grid = g_num_sms * per_sm;
    if (max_blocks > 0 && grid > max_blocks) grid = max_blocks;
    tail_kernel<N, G><<<grid, bt, smem, s>>>(L, tb);
    return cudaGetLastError();
}

cudaError_t launch_tail(const TrackLaunch &L, int max_blocks, cudaStream_t s)
{
    device_limits();
    switch (L.tab.n) {
    case 1: return launch_tail_n<1, 8>(L, max_blocks, s);
    case 2: return launch_tail_n<2, 8>(L, max_blocks, s);
    case 3: return launch_tail_n<3, 8>(L, max_blocks, s);
    case 4: return launch_tail_n<4, 8>(L, max_blocks, s);
    case 5: return launch_tail_n<5, 8>(L, max_blocks, s);
    case 6: return launch_tail_n<6, 8>(L, max_blocks, s);
    case 7: return launch_tail_n<7, 8>(L, max_blocks, s);
    case 8: return launch_tail_n<8, 8>(L, max_blocks, s);
    case 9: return launch_tail_n<9, 16>(L, max_blocks, s);
    case 10: return launch_tail_n<10, 16>(L, max_blocks, s);
    case 11: return launch_tail_n<11, 16>(L, max_blocks, s);
    case 12: return launch_tail_n<12, 16>(L, max_blocks, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace phc
