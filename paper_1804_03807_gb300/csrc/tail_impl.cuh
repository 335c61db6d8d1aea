// tail_impl.cuh -- a path tracked by a group of G threads (the device code of
// the tail kernels of track_tail.cu and of the grouped polyhedral tracker of
// track_poly.cu).
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
#pragma once
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


// The coefficients of a homotopy with coefficients linear in t (one
// coefficient set of a table): c0 + t c1 in H and H_x; in the right-hand
// side c1 (H_t) or the same c0 + t c1 (H).
struct LinearCoef {
    const double2 *C0, *C1;
    __device__ __forceinline__ double diverge_bound(const phc_opts &o) const { return o.diverge_norm; }
    __device__ __forceinline__ void operator()(int q, double te, bool dt, double2 &ct, double2 &cr)
    {
        const double2 c0 = C0[q], c1 = C1[q];
        ct = make_double2(fma(te, c1.x, c0.x), fma(te, c1.y, c0.y));
        cr = dt ? c1 : ct;
    }
};

// Tracks one path to its end with the G lanes of a group (base: the group's
// slots; coef(q, t, dt, ct, cr): term q's coefficient at t in H and H_x, and
// in the right-hand side, H_t when dt, else H; coef.diverge_bound(o): the
// norm beyond which the path counts as diverged).  The path starts from the
// state in hd (a handed-off path, or a fresh one: t = 0, counters 0).  At the
// end every lane calls finish(x0r, rec, units): lane r < N holds x_r, lane 0
// the statistics record, units = the units run here.
template <int N, int G, typename Coef, typename Finish>
__device__ __forceinline__ void tail_path(const Handoff &hd, const SmTab &tb, const TailPlan &plan, Coef coef,
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
            double2 ct, cr;
            coef(qq, te, dt, ct, cr);
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
            if (nx > coef.diverge_bound(o)) {
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

}  // namespace phc
