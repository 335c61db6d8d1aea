// track_tail.cu -- the tail kernel: G threads per path.
//
// When most lanes of a tracking launch have run out of paths, the remaining
// paths leave the one-thread-per-path kernel at the start of a step (see the
// hand-off in track_impl.cuh) and continue here with a group of G lanes per
// path, so that a long path no longer runs at the speed of one thread that
// shares an FP64 pipe with a mostly empty warp.  One evaluate+factor+solve
// unit of a path:
//   evaluation, phase A: the lanes take the terms (heaviest first) and run
//     add_term into a StoreSink -- the prefix and suffix products and the
//     coefficient of the right-hand side, kept in the group's term store;
//   evaluation, phase B: the lanes take the entries of H_x and of the
//     right-hand side (longest first) and add up each entry's pieces in the
//     order of the table, with the operations AccumSink would have used;
//   LU: one column at a time; pivot search by a butterfly arg-max (first row
//     on ties, as the one-thread loop), the row swap by columns, the trailing
//     update spread over all lanes;
//   solves: lane r owns row r (forward over ascending, back substitution over
//     descending columns, as lu_solve).
// Every value is computed by exactly the operations, in exactly the order,
// of the one-thread kernel, and the scalars of the step logic are reduced
// with exact operations (max, and), so a path ends with the same bits
// whichever kernel finishes it.
#include "track_impl.cuh"

namespace phc {

// Smallest power of two >= N: the lanes that hold rows of the group.
template <int N>
__host__ __device__ constexpr int rows_pow2()
{
    return N <= 1 ? 1 : N <= 2 ? 2 : N <= 4 ? 4 : N <= 8 ? 8 : 16;
}

// Maximum over the group of non-negative, non-NaN doubles held by its first
// P2 lanes, in every lane.  The bit pattern of a non-negative double orders
// like its value, so the comparisons are integer ones (the FP64 pipe, which
// bounds these kernels, is spared); the result is the same maximum.
template <int G, int P2>
__device__ __forceinline__ double gmax(double v, unsigned mask)
{
    unsigned long long k = (unsigned long long)__double_as_longlong(v);
#pragma unroll
    for (int o = P2 / 2; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(mask, k, o, G);
        k = (w > k) ? w : k;
    }
    return __longlong_as_double((long long)__shfl_sync(mask, k, 0, G));
}

// add_term's pieces of one term, kept in the term's slots of the group's
// store: (p_j, s_j) pairs for j = 0..k-2, then d, x^a and cr (2k + 1 slots).
struct StoreSink {
    double2 *s;
    int k;
    __device__ __forceinline__ void put_prefix(int j, double2 p) { s[2 * j] = p; }
    __device__ __forceinline__ double2 get_prefix(int j) const { return s[2 * j]; }
    __device__ __forceinline__ void last(int, double2 d) { s[2 * (k - 1)] = d; }
    __device__ __forceinline__ void deriv(int j, int, double2 pj, double2 suf)
    {
        s[2 * j] = pj;
        s[2 * j + 1] = suf;
    }
    __device__ __forceinline__ void rhs(double2 cr, double2 mono)
    {
        s[2 * k - 1] = mono;
        s[2 * k] = cr;
    }
};

// Contributions to an entry of H_x or of the right-hand side: slot | kind << 14.
enum : uint16_t { PIECE_FMA = 0, PIECE_ADD = 1, PIECE_RHS = 2 };

// Per-block plan of the two evaluation phases, built from the staged table:
// the term store layout, the order in which lanes take terms and entries,
// and each entry's pieces in table order.  Sizes in tail_plan_bytes.
struct TailPlan {
    uint16_t *tslot;   // [T] first store slot of term q
    uint16_t *torder;  // [T] terms, largest support first
    uint16_t *eoff;    // [E + 1] pieces of entry e: elist[eoff[e] .. eoff[e + 1])
    uint16_t *elist;   // [n_ve + T]
    uint16_t *eorder;  // [E] entries, most pieces first
};


template <int N>
static __device__ TailPlan plan_layout(const SmTab &tb, char *region)
{
    constexpr int E = N * N + N;
    const int T = tb.n_terms;
    TailPlan p;
    p.tslot = reinterpret_cast<uint16_t *>(region);
    p.torder = p.tslot + T;
    p.eoff = p.torder + T;
    p.elist = p.eoff + (E + 1);
    int n_pieces = 0;
    for (int q = 0; q < T; q++) n_pieces += tb.terms[q].k + 1;
    p.eorder = p.elist + n_pieces;
    return p;
}

// Fills the plan (one thread; the caller synchronises).
template <int N>
static __device__ void plan_fill(const SmTab &tb, const TailPlan &p)
{
    constexpr int E = N * N + N;
    const int T = tb.n_terms;
    uint16_t *cnt = p.eorder;  // scratch: E counters, then the entry order
    int slot = 0, kmax = 0;
    for (int e = 0; e < E; e++) cnt[e] = 0;
    for (int q = 0; q < T; q++) {
        const TermRec r = tb.terms[q];
        p.tslot[q] = (uint16_t)slot;
        slot += r.k ? 2 * r.k + 1 : 1;
        kmax = r.k > kmax ? r.k : kmax;
        for (int j = 0; j < r.k; j++) cnt[r.eq * N + tb.vars[r.off + j]]++;
        cnt[N * N + r.eq]++;
    }
    // terms by decreasing support size (stable)
    int w = 0;
    for (int k = kmax; k >= 0; k--)
        for (int q = 0; q < T; q++)
            if (tb.terms[q].k == k) p.torder[w++] = (uint16_t)q;
    int acc = 0, lmax = 0;
    for (int e = 0; e < E; e++) {
        p.eoff[e] = (uint16_t)acc;
        acc += cnt[e];
        lmax = cnt[e] > lmax ? cnt[e] : lmax;
        cnt[e] = 0;
    }
    p.eoff[E] = (uint16_t)acc;
    // pieces in table order; within a term the columns in the order add_term emits them
    for (int q = 0; q < T; q++) {
        const TermRec r = tb.terms[q];
        const int b = p.tslot[q], k = r.k;
        if (k) {
            for (int j = k - 1; j >= 0; j--) {
                const int e = r.eq * N + tb.vars[r.off + j];
                const uint16_t v = (j == k - 1) ? (uint16_t)((b + 2 * (k - 1)) | (PIECE_ADD << 14))
                                                : (uint16_t)((b + 2 * j) | (PIECE_FMA << 14));
                p.elist[p.eoff[e] + cnt[e]++] = v;
            }
            const int e = N * N + r.eq;
            p.elist[p.eoff[e] + cnt[e]++] = (uint16_t)((b + 2 * k - 1) | (PIECE_RHS << 14));
        } else {
            const int e = N * N + r.eq;
            p.elist[p.eoff[e] + cnt[e]++] = (uint16_t)(b | (PIECE_ADD << 14));
        }
    }
    // entries by decreasing number of pieces (overwrites the counters)
    w = 0;
    for (int l = lmax; l >= 0; l--)
        for (int e = 0; e < E; e++)
            if (p.eoff[e + 1] - p.eoff[e] == l) p.eorder[w++] = (uint16_t)e;
}


// Tracks one handed-off path to its end with the G lanes of a group (base:
// the group's slots; coef_sys: the coefficient set of a batch table).  At
// the end every lane calls finish(x0r, rec, units): lane r < N holds x_r,
// lane 0 the statistics record, units = the units run here.
template <int N, int G, typename Finish>
__device__ __forceinline__ void tail_path(const Handoff &hd, const SmTab &tb, const TailPlan &plan, int coef_sys,
                                          double2 *base, const phc_opts &o, int r, unsigned gmask, Finish &&finish)
{
    constexpr int E = N * N + N;
    constexpr int P2 = rows_pow2<N>();
    const int T = tb.n_terms;
    double2 *xe = base;          // [N]
    double2 *R = base + N;       // [N]
    double2 *J = base + 2 * N;   // [N][N]
    double2 *store = base + 2 * N + N * N;  // add_term pieces of every term
    const bool own = r < N;
    double t = hd.t, h = hd.h, next_s = hd.next_s;
    double r0 = hd.r0, r1 = hd.r1, r2 = hd.r2, r3 = hd.r3, r4 = hd.r4;
    const int sys = hd.sys;
    int streak = hd.streak, steps = hd.steps, since_ck = hd.since_ck, nck = hd.nck;
    int n_acc = hd.n_acc, n_rej = hd.n_rej, n_newt = hd.n_newt, n_solve = hd.n_solve;
    const int n_f32 = hd.n_f32;
    double2 x0r = own ? hd.x0[r] : make_double2(0.0, 0.0);
    double2 accr = make_double2(0.0, 0.0), solr = make_double2(0.0, 0.0);
    double he = 0.0, t1 = 0.0, te = 0.0, prev = 0.0;
    int phase = 0, it = 0;
    const double2 *C0 = tb.c0 + (size_t)coef_sys * tb.n_terms, *C1 = tb.c1 + (size_t)coef_sys * tb.n_terms;

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
        // ---------------------------------------------- evaluation, phase A: the terms' pieces
        const bool dt = phase < 4;
        for (int i = r; i < T; i += G) {
            const int qq = plan.torder[i];
            const TermRec rec = tb.terms[qq];
            const double2 c0 = C0[qq], c1 = C1[qq];
            const double2 ct = make_double2(fma(te, c1.x, c0.x), fma(te, c1.y, c0.y));
            const double2 cr = dt ? c1 : ct;
            double2 *ts = store + plan.tslot[qq];
            if (rec.k == 0) {
                ts[0] = cr;
            } else {
                StoreSink sink{ts, rec.k};
                add_term<double2>(rec, tb.vars + rec.off, tb.exps + rec.off, ct, cr, xe, 1, sink);
            }
        }
        __syncwarp(gmask);
        // ---------------------------------------------- evaluation, phase B: the entries, pieces in table order
        for (int i = r; i < E; i += G) {
            const int e = plan.eorder[i];
            double2 a = make_double2(0.0, 0.0);
            for (int m = plan.eoff[e]; m < plan.eoff[e + 1]; m++) {
                const uint16_t w = plan.elist[m];
                const double2 *pc = store + (w & 0x3fff);
                const int kind = w >> 14;
                if (kind == PIECE_FMA) a = cfma(pc[0], pc[1], a);
                else if (kind == PIECE_ADD) a = cadd(a, pc[0]);
                else a = cfma(pc[1], pc[0], a);
            }
            if (e < N * N) J[e] = a;
            else R[e - N * N] = a;
        }
        __syncwarp(gmask);
        // ---------------------------------------------- LU (as lu_factor<N, double2>)
        bool ok = true;
        int perm[N];
#pragma unroll
        for (int k = 0; k < N; k++) {
            const double vk = abs1(J[k * N + k]);
            // candidates: rows i > k with a larger |.|_1 (the first on ties);
            // keyed by the bit pattern of |.|_1 (integer compares), a row
            // without a candidate (or with a NaN) by 0 and the index N
            unsigned long long key = 0ull;
            int bi = N;
            if (own && r > k) {
                const double a = abs1(J[r * N + k]);
                if (a == a) {
                    key = (unsigned long long)__double_as_longlong(a);
                    bi = r;
                }
            }
#pragma unroll
            for (int off = P2 / 2; off > 0; off >>= 1) {
                const unsigned long long ok2 = __shfl_xor_sync(gmask, key, off, G);
                const int oi = __shfl_xor_sync(gmask, bi, off, G);
                if (ok2 > key || (ok2 == key && oi < bi)) {
                    key = ok2;
                    bi = oi;
                }
            }
            key = __shfl_sync(gmask, key, 0, G);
            bi = __shfl_sync(gmask, bi, 0, G);
            const double bv = __longlong_as_double((long long)key);
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
            if (own && r > k) J[r * N + k] = cmul(J[r * N + k], inv);
            __syncwarp(gmask);
            // trailing update J[i][j] -= l_i J[k][j], i, j > k, spread over the group
            const int M = N - 1 - k;
            if (M > 0) {
                for (int m = r; m < M * M; m += G) {
                    const int i = k + 1 + m / M, j = k + 1 + m % M;
                    J[i * N + j] = cfms(J[i * N + j], J[i * N + k], J[k * N + j]);
                }
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
            const double d = fin ? gmax<G, P2>(a, gmask) : NAN;
            const double nx = fin ? gmax<G, P2>(c, gmask) : NAN;
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
            const double nx = gmax<G, P2>(own ? absinf(x0r) : 0.0, gmask);
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
    phc_path_stats rec{};
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
    }
    finish(x0r, rec, n_solve - hd.n_solve);
    __syncwarp(gmask);
}

template <int N, int G>
__global__ void __launch_bounds__(128) tail_kernel(const TrackLaunch L, size_t table_bytes, size_t plan_bytes)
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
    const int64_t np = L.n_paths;
    const unsigned long long n_hand = *reinterpret_cast<volatile const unsigned long long *>(L.handoff_n);
    for (;;) {
        unsigned long long slot = 0;
        if (r == 0) slot = atomicAdd(L.tail_q, 1ull);
        slot = __shfl_sync(gmask, slot, 0, G);
        if (slot >= n_hand) break;
        const Handoff &hd = L.handoff[slot];
        const int64_t q = hd.q;
        tail_path<N, G>(hd, tb, plan, hd.sys, base, L.o, r, gmask,
                        [&](double2 x0r, const phc_path_stats &rec, int units) {
                            if (r < N) L.x_out[(int64_t)r * np + q] = x0r;
                            if (r == 0) {
                                L.stats[q] = rec;
                                atomicAdd(L.tail_units, (unsigned long long)units);
                            }
                        });
    }
}

// classify_one for one lane, out of line: it needs many registers, the
// tracking loop of the tail kernel does not.
template <int N>
__device__ __noinline__ int8_t classify_lane(const SmTab &tb, const ThreadArrays &A, phc_path_stats &rec,
                                             const phc_opts &o)
{
    return classify_one<N>(tb, A, rec, o, 1);
}

// The multi-system tail: one warp per path; each warp stages the table and
// builds the plan of the path's system in its own region (again only when
// the system changes), and classifies the endpoint (in lane 0, with
// classify_one, as the multi-system tracker does inline).
template <int N>
__global__ void __launch_bounds__(128) tail_multi_kernel(const TrackLaunch L, size_t region_bytes,
                                                         size_t table_cap, size_t plan_cap)
{
    extern __shared__ __align__(16) char smem[];
    constexpr int G = 32;
    const int r = threadIdx.x & 31;
    char *region = smem + (size_t)(threadIdx.x >> 5) * region_bytes;
    double2 *base = reinterpret_cast<double2 *>(region + table_cap + plan_cap);
    const unsigned long long n_hand = *reinterpret_cast<volatile const unsigned long long *>(L.handoff_n);
    int cur = -1;
    SmTab tb{};
    TailPlan plan{};
    for (;;) {
        unsigned long long slot = 0;
        if (r == 0) slot = atomicAdd(L.tail_q, 1ull);
        slot = __shfl_sync(0xffffffffu, slot, 0);
        if (slot >= n_hand) break;
        const Handoff &hd = L.handoff[slot];
        const int ws = hd.sys;
        const SysDesc &d = L.multi[ws];
        if (ws != cur) {
            __syncwarp();
            tb = stage_table_warp(d.tab, region);
            plan = plan_layout<N>(tb, region + table_cap);
            if (r == 0) plan_fill<N>(tb, plan);
            __syncwarp();
            cur = ws;
        }
        const int64_t q = hd.q;
        tail_path<N, G>(hd, tb, plan, 0, base, L.o, r, 0xffffffffu,
                        [&](double2 x0r, const phc_path_stats &rec0, int units) {
                            // classification arrays over the group's slots, stride 1
                            ThreadArrays A;
                            A.xe = base;
                            A.R = A.xe + N;
                            A.P = A.R + N;
                            A.X = A.P;
                            A.J = A.P + N;
                            A.S = A.J + N * N;
                            if (r < N) {
                                A.xe[r] = x0r;
                                d.x_out[(int64_t)r * d.n_paths + q] = x0r;
                            }
                            __syncwarp();
                            if (r == 0) {
                                phc_path_stats rec = rec0;
                                rec.system = 0;
                                const int8_t c = classify_lane<N>(tb, A, rec, L.o);
                                rec.system = ws;
                                d.stats[q] = rec;
                                d.cls_out[q] = c;
                                atomicAdd(L.tail_units, (unsigned long long)units);
                            }
                            __syncwarp();
                        });
    }
}

// The pipelined tail: one warp per path of a pipelined launch.  A path
// handed off in the top stage ends there, is classified (lane 0,
// classify_one on the top table) and, when regular with z_k != 0, starts
// the cascade stage from its endpoint in the same warp, exactly as the
// pipelined tracker continues it in the same lane.
template <int N>
__global__ void __launch_bounds__(128) tail_pipe_kernel(const TrackLaunch L, size_t t1_bytes, size_t t2_bytes,
                                                        size_t p1_bytes, size_t p2_bytes, int group_slots)
{
    extern __shared__ __align__(16) char smem[];
    const SmTab tb1 = stage_table(L.tab, smem);
    const SmTab tb2 = stage_table(L.tab2, smem + t1_bytes);
    const TailPlan plan1 = plan_layout<N>(tb1, smem + t1_bytes + t2_bytes);
    const TailPlan plan2 = plan_layout<N>(tb2, smem + t1_bytes + t2_bytes + p1_bytes);
    if (threadIdx.x == 0) {
        plan_fill<N>(tb1, plan1);
        plan_fill<N>(tb2, plan2);
    }
    __syncthreads();
    constexpr int G = 32;
    constexpr unsigned FULL = 0xffffffffu;
    const int r = threadIdx.x & 31;
    constexpr int HS = (int)((sizeof(Handoff) + 15) / 16);
    double2 *base = reinterpret_cast<double2 *>(smem + t1_bytes + t2_bytes + p1_bytes + p2_bytes) +
                    (size_t)(threadIdx.x >> 5) * (group_slots + HS);
    Handoff *hs = reinterpret_cast<Handoff *>(base + group_slots);  // the fresh cascade-stage start
    const phc_opts &o = L.o;
    const int64_t np = L.n_paths;
    const unsigned long long n_hand = *reinterpret_cast<volatile const unsigned long long *>(L.handoff_n);
    ThreadArrays A;  // one-lane classification arrays over the group's slots (stride 1)
    A.xe = base;
    A.R = A.xe + N;
    A.P = A.R + N;
    A.X = A.P;
    A.J = A.P + N;
    A.S = A.J + N * N;
    for (;;) {
        unsigned long long slot = 0;
        if (r == 0) slot = atomicAdd(L.tail_q, 1ull);
        slot = __shfl_sync(FULL, slot, 0);
        if (slot >= n_hand) break;
        const Handoff *cur = &L.handoff[slot];
        const int64_t q = cur->q;
        int stage = cur->stage;
        for (;;) {
            int cont = 0;
            const SmTab &tb = stage ? tb2 : tb1;
            tail_path<N, G>(*cur, tb, stage ? plan2 : plan1, 0, base, o, r, FULL,
                            [&](double2 x0r, const phc_path_stats &rec0, int units) {
                                if (r < N) A.xe[r] = x0r;
                                __syncwarp();
                                if (r == 0) {
                                    phc_path_stats rec = rec0;
                                    const int8_t c = classify_lane<N>(tb, A, rec, o);
                                    atomicAdd(L.tail_units, (unsigned long long)units);
                                    if (stage == 0) {
                                        for (int j = 0; j < N; j++) L.x_out[(int64_t)j * np + q] = A.xe[j];
                                        L.stats[q] = rec;
                                        L.cls_out[q] = c;
                                        if (c == PHC_REGULAR &&
                                            absinf(A.xe[N - 1]) > o.slack_tol * (1.0 + rec.norm_x)) {
                                            cont = 1;
                                        } else {
                                            L.cls_out2[q] = -1;
                                        }
                                    } else {
                                        double nx = 0.0;
                                        for (int j = 0; j < N - 1; j++) {
                                            L.x_out2[(int64_t)j * np + q] = A.xe[j];
                                            const double a = absinf(A.xe[j]);
                                            if (!(a <= nx)) nx = a;
                                        }
                                        L.stats2[q] = rec;
                                        L.cls_out2[q] = c;
                                        L.slack_zero2[q] =
                                            L.has_next_slack ? (absinf(A.xe[N - 2]) <= o.slack_tol * (1.0 + nx)) : 0;
                                    }
                                }
                                cont = __shfl_sync(FULL, cont, 0);
                                if (cont) {
                                    // the state the pipelined tracker gives a fresh path
                                    if (r < N) hs->x0[r] = x0r;
                                    if (r == 0) {
                                        hs->t = 0.0;
                                        hs->h = o.h_init;
                                        hs->next_s = 0.1;
                                        hs->nx0 = 0.0;
                                        hs->r0 = hs->r1 = hs->r2 = hs->r3 = hs->r4 = 0.0;
                                        hs->q = q;
                                        hs->sys = 0;
                                        hs->streak = hs->steps = hs->since_ck = hs->nck = 0;
                                        hs->n_acc = hs->n_rej = hs->n_newt = hs->n_solve = hs->n_f32 = 0;
                                        hs->stage = 1;
                                    }
                                }
                                __syncwarp();
                            });
            if (!cont) break;
            stage = 1;
            cur = hs;
        }
    }
}

template <int N>
static cudaError_t launch_tail_pipe_n(const TrackLaunch &L_in, int max_blocks, cudaStream_t s)
{
    TrackLaunch L = L_in;
    L.tab.coef_smem = L.tab2.coef_smem = 1;
    const size_t t1 = table_smem_bytes(L.tab), t2 = table_smem_bytes(L.tab2);
    const size_t p1 = tail_plan_bytes(N, L.tab.n_terms, L.tab.n_ve), p2 = tail_plan_bytes(N, L.tab2.n_terms, L.tab2.n_ve);
    const int S1 = tail_store_slots(L.tab.n_terms, L.tab.n_ve), S2 = tail_store_slots(L.tab2.n_terms, L.tab2.n_ve);
    const int gs = tail_group_slots(N, S1 > S2 ? S1 : S2);
    const size_t per_warp = (size_t)(gs + (sizeof(Handoff) + 15) / 16) * sizeof(double2);
    int warps = 4;
    while (warps > 1 && t1 + t2 + p1 + p2 + warps * per_warp > (size_t)g_smem_optin) warps /= 2;
    const size_t smem = t1 + t2 + p1 + p2 + warps * per_warp;
    if (smem > (size_t)g_smem_optin) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(tail_pipe_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tail_pipe_kernel<N>, warps * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int grid = g_num_sms * per_sm;
    if (max_blocks > 0 && grid > max_blocks) grid = max_blocks;
    tail_pipe_kernel<N><<<grid, warps * 32, smem, s>>>(L, t1, t2, p1, p2, gs);
    return cudaGetLastError();
}

cudaError_t launch_tail_pipe(const TrackLaunch &L, int max_blocks, cudaStream_t s)
{
    device_limits();
#define PHC_CALL_TAILP(NN) launch_tail_pipe_n<NN>(L, max_blocks, s)
    PHC_DISPATCH_N(L.tab.n, PHC_CALL_TAILP)
#undef PHC_CALL_TAILP
}

bool tail_pipe_supported(const DevTables &t1_in, const DevTables &t2_in)
{
    device_limits();
    const int n = t1_in.n;
    if (n < 2 || n > PHC_MAX_VARS) return false;
    DevTables t1 = t1_in, t2 = t2_in;
    t1.coef_smem = t2.coef_smem = 1;
    const int S1 = tail_store_slots(t1.n_terms, t1.n_ve), S2 = tail_store_slots(t2.n_terms, t2.n_ve);
    if (S1 >= (1 << 14) || S2 >= (1 << 14)) return false;
    const size_t need = table_smem_bytes(t1) + table_smem_bytes(t2) + tail_plan_bytes(n, t1.n_terms, t1.n_ve) +
                        tail_plan_bytes(n, t2.n_terms, t2.n_ve) +
                        (size_t)(tail_group_slots(n, S1 > S2 ? S1 : S2) + (sizeof(Handoff) + 15) / 16) *
                            sizeof(double2);
    return need <= (size_t)g_smem_optin;
}

template <int N, int G>
static cudaError_t launch_tail_n(const TrackLaunch &L_in, int max_blocks, cudaStream_t s)
{
    TrackLaunch L = L_in;
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
    cudaError_t e = cudaFuncSetAttribute(tail_kernel<N, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tail_kernel<N, G>, bt, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int grid = g_num_sms * per_sm;
    if (max_blocks > 0 && grid > max_blocks) grid = max_blocks;
    tail_kernel<N, G><<<grid, bt, smem, s>>>(L, tb, pb);
    return cudaGetLastError();
}

bool tail_supported(const DevTables &t)
{
    device_limits();
    const int n = t.n;
    if (n < 1 || n > PHC_MAX_VARS) return false;
    const int S = tail_store_slots(t.n_terms, t.n_ve);
    if (S >= (1 << 14)) return false;  // slot numbers are 14-bit
    DevTables u = t;
    u.coef_smem = 0;
    const size_t need = table_smem_bytes(u) + tail_plan_bytes(n, t.n_terms, t.n_ve) +
                        (size_t)tail_group_slots(n, S) * sizeof(double2);
    return need <= (size_t)g_smem_optin;
}

// opts.tail_threads picks G: 8 (N <= 8 only), 16 or 32; 0 = 32.
#define PHC_TAIL_CASE(NN)                                                                                             \
    case NN:                                                                                                          \
        if (group == 8 && (NN) <= 8) return launch_tail_n<NN, ((NN) <= 8 ? 8 : 16)>(L, max_blocks, s);              \
        if (group == 16) return launch_tail_n<NN, 16>(L, max_blocks, s);                                             \
        return launch_tail_n<NN, 32>(L, max_blocks, s);

cudaError_t launch_tail(const TrackLaunch &L, int max_blocks, cudaStream_t s)
{
    device_limits();
    const int group = L.o.tail_threads;
    switch (L.tab.n) {
        PHC_TAIL_CASE(1)
        PHC_TAIL_CASE(2)
        PHC_TAIL_CASE(3)
        PHC_TAIL_CASE(4)
        PHC_TAIL_CASE(5)
        PHC_TAIL_CASE(6)
        PHC_TAIL_CASE(7)
        PHC_TAIL_CASE(8)
        PHC_TAIL_CASE(9)
        PHC_TAIL_CASE(10)
        PHC_TAIL_CASE(11)
        PHC_TAIL_CASE(12)
    default: return cudaErrorInvalidValue;
    }
}
#undef PHC_TAIL_CASE

template <int N>
static cudaError_t launch_tail_multi_n(const TrackLaunch &L, const TailMultiSizes &z, int max_blocks, cudaStream_t s)
{
    const size_t region = z.table_cap + z.plan_cap + (size_t)z.group_slots * sizeof(double2);
    int warps = 4;
    while (warps > 1 && warps * region > (size_t)g_smem_optin) warps /= 2;
    if (warps * region > (size_t)g_smem_optin) return cudaErrorInvalidConfiguration;
    const size_t smem = warps * region;
    cudaError_t e =
        cudaFuncSetAttribute(tail_multi_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tail_multi_kernel<N>, warps * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int grid = g_num_sms * per_sm;
    if (max_blocks > 0 && grid > max_blocks) grid = max_blocks;
    tail_multi_kernel<N><<<grid, warps * 32, smem, s>>>(L, region, z.table_cap, z.plan_cap);
    return cudaGetLastError();
}

bool tail_multi_supported(const TailMultiSizes &z)
{
    device_limits();
    return z.max_store < (1 << 14) &&  // slot numbers are 14-bit
           z.table_cap + z.plan_cap + (size_t)z.group_slots * sizeof(double2) <= (size_t)g_smem_optin;
}

cudaError_t launch_tail_multi(const TrackLaunch &L, int n, const TailMultiSizes &z, int max_blocks, cudaStream_t s)
{
    device_limits();
#define PHC_CALL_TAILM(NN) launch_tail_multi_n<NN>(L, z, max_blocks, s)
    PHC_DISPATCH_N(n, PHC_CALL_TAILM)
#undef PHC_CALL_TAILM
}

}  // namespace phc
