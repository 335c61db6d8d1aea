// mixed_cells.cpp -- fine mixed cells of a lifted system of supports, and the
// per-cell data of its polyhedral homotopy (host code).
//
// Section 2.2: a random coefficient start system is solved by polyhedral
// homotopies, one per mixed cell of a mixed subdivision of the Newton
// polytopes; a cell of volume V starts V paths, and the cells are produced one
// after the other while the paths of the cells already made are tracked
// (Figure 2).  Definitions used here:
//   supports A_i = the exponent vectors of equation i's terms; an integer
//   lifting w (one value per term).  A fine mixed cell picks {a_i, b_i} in
//   every A_i and has an inner normal v in Q^n with, for every i,
//       <a, v> + w(a) = beta_i  on the pair,  > beta_i  on the rest of A_i.
//   Its volume is |det D|, D the integer matrix with rows b_i - a_i.
//
// Enumeration: depth first over the equations, at every node the equation
// with the fewest edges related to all edges chosen so far (a node where one
// has none is a dead end).  A pair of the next equation must (1) be a lower edge of its own
// lifted support, (2) be compatible with every pair chosen so far (a relation
// table of two-pair feasibility problems, solved once) and (3) keep the
// problem of all pairs chosen so far feasible.  Complete choices are checked
// exactly in 128-bit integer arithmetic.  The feasibility problems are linear
// programs in double precision that only drop choices whose optimum is clearly
// infeasible, so rounding can cost time but never a cell.  The edge tests,
// the relation table and the subtrees below the first few equations run on
// the host's threads; the cells come out in the order of the sequential
// search whatever the number of threads.
//
// Feasibility of the chosen pairs P: maximize tau over (v, tau) with
//   <a - b, v> = w(b) - w(a)                    for every pair (a, b) in P,
//   <c - a, v> + w(c) - w(a) >= tau             for every other point c of a
//                                               chosen support,   tau <= 1;
// strictly feasible when the optimum is positive.  It is solved through its
// dual, min (sum_c (w(c)-w(a)) y_c + y_0 + sum_P (w(b)-w(a)) mu_P) subject to
// sum_c y_c (a - c) + sum_P mu_P (a - b) = 0, sum_c y_c + y_0 = 1, y >= 0
// (mu free, split in two), a standard-form problem with n + 1 rows that the
// dense two-phase simplex below (Bland's rule) solves; an unbounded dual
// means inconsistent equalities.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <condition_variable>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "phc_internal.h"

namespace phc {

int set_error(int code, const char *msg);

namespace {

typedef __int128 i128;

// ------------------------------------------------------------------ linear programming

// min cost.y subject to M y = b (b >= 0), y >= 0; M is R x C row-major.
// Returns 0 (optimal, *val), 1 (unbounded), 2 (infeasible), 3 (no answer
// within the iteration limit).
int simplex(int R, int C, const double *M, const double *b, const double *cost, double *val)
{
    const int W = C + R + 1;
    thread_local std::vector<double> T;
    thread_local std::vector<int> basis;
    T.assign((size_t)(R + 1) * W, 0.0);
    basis.assign(R, 0);
    double cmax = 0.0;
    for (int j = 0; j < C; j++) cmax = std::max(cmax, std::fabs(cost[j]));
    for (int i = 0; i < R; i++) {
        for (int j = 0; j < C; j++) T[(size_t)i * W + j] = M[(size_t)i * C + j];
        T[(size_t)i * W + C + i] = 1.0;
        T[(size_t)i * W + W - 1] = b[i];
        basis[i] = C + i;
    }
    double *obj = &T[(size_t)R * W];
    auto pivot = [&](int r, int e) {
        double *rr = &T[(size_t)r * W];
        const double p = rr[e];
        for (int j = 0; j < W; j++) rr[j] /= p;
        for (int i = 0; i <= R; i++) {
            if (i == r) continue;
            double *ri = &T[(size_t)i * W];
            const double f = ri[e];
            if (f == 0.0) continue;
            for (int j = 0; j < W; j++) ri[j] -= f * rr[j];
        }
        basis[r] = e;
    };
    // returns 0 optimal, 1 unbounded, 3 iteration limit; the most negative
    // reduced cost enters, after 4 (R + C) pivots the first negative one
    // (Bland's rule, which cannot cycle)
    auto run = [&](int allow, double eps_cost) -> int {
        const int limit = 64 * (R + C) + 256, bland_after = 4 * (R + C);
        for (int it = 0; it < limit; it++) {
            int e = -1;
            if (it < bland_after) {
                double best = -eps_cost;
                for (int j = 0; j < allow; j++)
                    if (obj[j] < best) {
                        best = obj[j];
                        e = j;
                    }
            } else {
                for (int j = 0; j < allow; j++)
                    if (obj[j] < -eps_cost) {
                        e = j;
                        break;
                    }
            }
            if (e < 0) return 0;
            int r = -1;
            double best = 0.0;
            for (int i = 0; i < R; i++) {
                const double a = T[(size_t)i * W + e];
                if (a <= 1e-11) continue;
                const double ratio = T[(size_t)i * W + W - 1] / a;
                if (r < 0 || ratio < best - 1e-13 || (ratio <= best + 1e-13 && basis[i] < basis[r])) {
                    r = i;
                    best = ratio;
                }
            }
            if (r < 0) return 1;
            pivot(r, e);
        }
        return 3;
    };
    // phase 1: minimise the sum of the artificial variables
    for (int j = 0; j < C; j++) {
        double s = 0.0;
        for (int i = 0; i < R; i++) s += T[(size_t)i * W + j];
        obj[j] = -s;
    }
    {
        double s = 0.0;
        for (int i = 0; i < R; i++) s += b[i];
        obj[W - 1] = -s;
    }
    int rc = run(C, 1e-10);
    if (rc == 3) return 3;
    if (-obj[W - 1] > 1e-9) return 2;
    for (int i = 0; i < R; i++) {
        if (basis[i] < C) continue;
        int e = -1;
        for (int j = 0; j < C; j++)
            if (std::fabs(T[(size_t)i * W + j]) > 1e-9) {
                e = j;
                break;
            }
        if (e >= 0) pivot(i, e);  // otherwise the row is redundant; its artificial stays at 0
    }
    // phase 2
    for (int j = 0; j < W; j++) obj[j] = j < C ? cost[j] : 0.0;
    for (int i = 0; i < R; i++) {
        const double cb = basis[i] < C ? cost[basis[i]] : 0.0;
        if (cb == 0.0) continue;
        for (int j = 0; j < W; j++) obj[j] -= cb * T[(size_t)i * W + j];
    }
    rc = run(C, 1e-10 * (1.0 + cmax));
    if (rc != 0) return rc;
    *val = -obj[W - 1];
    return 0;
}

struct Lifted {
    int n = 0;
    std::vector<int> off, m;                // per equation: first term, number of terms
    std::vector<int64_t> A;                 // [T][n] exponents
    std::vector<int64_t> w;                 // [T] lifting
    double wmax = 0.0;
    int64_t at(int t, int j) const { return A[(size_t)t * n + j]; }
};

struct Pair {
    int eq, a, b;  // global term indices a < b of equation eq
};

// Is the set of pairs strictly feasible (see the file comment)?  Leans to
// "yes" whenever the answer is not clear.
bool feasible(const Lifted &L, const Pair *P, int np)
{
    const int n = L.n;
    const int R = n + 1;
    thread_local std::vector<double> cols, cost, M, rhs;  // cols: column-major, C columns of R
    cols.clear();
    cost.clear();
    for (int p = 0; p < np; p++) {
        const int i = P[p].eq, a = P[p].a, b = P[p].b;
        for (int c = L.off[i]; c < L.off[i] + L.m[i]; c++) {
            if (c == a || c == b) continue;
            for (int j = 0; j < n; j++) cols.push_back((double)(L.at(a, j) - L.at(c, j)));
            cols.push_back(1.0);
            cost.push_back((double)(L.w[c] - L.w[a]));
        }
    }
    for (int j = 0; j < n; j++) cols.push_back(0.0);  // y_0 (tau <= 1)
    cols.push_back(1.0);
    cost.push_back(1.0);
    for (int p = 0; p < np; p++) {
        const int a = P[p].a, b = P[p].b;
        for (int s = 1; s >= -1; s -= 2) {
            for (int j = 0; j < n; j++) cols.push_back((double)(s * (L.at(a, j) - L.at(b, j))));
            cols.push_back(0.0);
            cost.push_back((double)(s * (L.w[b] - L.w[a])));
        }
    }
    const int C = (int)cost.size();
    M.resize((size_t)R * C);
    rhs.assign(R, 0.0);
    for (int c = 0; c < C; c++)
        for (int r = 0; r < R; r++) M[(size_t)r * C + c] = cols[(size_t)c * R + r];
    rhs[n] = 1.0;
    double val = 0.0;
    const int rc = simplex(R, C, M.data(), rhs.data(), cost.data(), &val);
    if (rc == 1 || rc == 2) return false;
    if (rc != 0) return true;
    return val > -1e-7 * (1.0 + L.wmax);
}

// The same dual problem kept along the depth-first search: a node's problem
// is its parent's with the columns of one more pair, so the parent's final
// basis stays feasible and the simplex continues from it (a few pivots)
// instead of starting over.  The state holds the columns in the current
// basis' coordinates (B^-1 M), B^-1 itself, B^-1 r, the reduced costs and
// the multipliers.
struct DualLP {
    int R = 0, C = 0;
    std::vector<double> A;     // column j at A[j * R ..]: B^-1 M_j
    std::vector<double> Binv;  // R x R row-major
    std::vector<double> rhs;   // B^-1 r
    std::vector<double> d;     // reduced costs of the real columns
    std::vector<double> cost;  // costs of the real columns
    std::vector<double> pi;    // multipliers c_B^T B^-1
    std::vector<int> basis;    // column of each row; -1 - k for the artificial of row k
    double z = 0.0, cmax = 0.0;
    int status = 0;            // 0 optimal, 1 unbounded, 2 infeasible, 3 no answer

    void pivot(int r, int e)
    {
        const double p = A[(size_t)e * R + r];
        // the entering column's multipliers, row r's taken out (0): the
        // update below then runs down whole columns, the memory order of A
        double fr[PHC_MAX_VARS + 1];
        for (int i = 0; i < R; i++) fr[i] = i == r ? 0.0 : A[(size_t)e * R + i];
        for (int k = 0; k < R; k++) Binv[(size_t)r * R + k] /= p;
        rhs[r] /= p;
        for (int j = 0; j < C; j++) {
            double *col = &A[(size_t)j * R];
            const double ar = col[r] / p;
            col[r] = ar;
            if (ar == 0.0) continue;
            for (int i = 0; i < R; i++) col[i] -= fr[i] * ar;
        }
        for (int i = 0; i < R; i++) {
            if (fr[i] == 0.0) continue;
            for (int k = 0; k < R; k++) Binv[(size_t)i * R + k] -= fr[i] * Binv[(size_t)r * R + k];
            rhs[i] -= fr[i] * rhs[r];
        }
        const double f = d[e];
        if (f != 0.0) {
            for (int j = 0; j < C; j++) d[j] -= f * A[(size_t)j * R + r];
            for (int k = 0; k < R; k++) pi[k] += f * Binv[(size_t)r * R + k];
            z += f * rhs[r];
        }
        basis[r] = e;
    }
    // Primal simplex on the reduced costs d (artificial columns never
    // enter): the most negative reduced cost enters (Dantzig), and after
    // 4 (R + C) pivots the first negative one (Bland's rule, which cannot
    // cycle).  0 optimal, 1 unbounded, 3 iteration limit, 4 the objective
    // of the (feasible) basis fell below z_stop: the minimum lies below it.
    int run(double eps, double z_stop = -INFINITY)
    {
        const int limit = 64 * (R + C) + 256, bland_after = 4 * (R + C);
        for (int it = 0; it < limit; it++) {
            int e = -1;
            if (it < bland_after) {
                double best = -eps;
                for (int j = 0; j < C; j++)
                    if (d[j] < best) {
                        best = d[j];
                        e = j;
                    }
            } else {
                for (int j = 0; j < C; j++)
                    if (d[j] < -eps) {
                        e = j;
                        break;
                    }
            }
            if (e < 0) return 0;
            int r = -1;
            double best = 0.0;
            for (int i = 0; i < R; i++) {
                const double a = A[(size_t)e * R + i];
                if (a <= 1e-11) continue;
                const double ratio = rhs[i] / a;
                const int bi = basis[i] >= 0 ? basis[i] : C + (-1 - basis[i]);
                const int br = r < 0 ? 0 : (basis[r] >= 0 ? basis[r] : C + (-1 - basis[r]));
                if (r < 0 || ratio < best - 1e-13 || (ratio <= best + 1e-13 && bi < br)) {
                    r = i;
                    best = ratio;
                }
            }
            if (r < 0) return 1;
            pivot(r, e);
            if (z < z_stop) return 4;
        }
        return 3;
    }
    // Appends an original column m (R entries) of cost c.
    void add_column(const double *m, double c)
    {
        A.resize((size_t)(C + 1) * R);
        double *a = &A[(size_t)C * R];
        double red = c;
        for (int i = 0; i < R; i++) {
            double s = 0.0;
            for (int k = 0; k < R; k++) s += Binv[(size_t)i * R + k] * m[k];
            a[i] = s;
            red -= pi[i] * m[i];
        }
        d.push_back(red);
        cost.push_back(c);
        cmax = std::max(cmax, std::fabs(c));
        C++;
    }
};

// The dual problem's columns of pair (i, a, b): one per other point c of
// support i, (a - c, 1) of cost w(c) - w(a), and the pair's equality as two
// columns +-(a - b, 0) of costs +-(w(b) - w(a)).
void pair_columns(const Lifted &L, const Pair &P, std::vector<double> &cols, std::vector<double> &costs)
{
    const int n = L.n, i = P.eq, a = P.a, b = P.b;
    for (int c = L.off[i]; c < L.off[i] + L.m[i]; c++) {
        if (c == a || c == b) continue;
        for (int j = 0; j < n; j++) cols.push_back((double)(L.at(a, j) - L.at(c, j)));
        cols.push_back(1.0);
        costs.push_back((double)(L.w[c] - L.w[a]));
    }
    for (int s = 1; s >= -1; s -= 2) {
        for (int j = 0; j < n; j++) cols.push_back((double)(s * (L.at(a, j) - L.at(b, j))));
        cols.push_back(0.0);
        costs.push_back((double)(s * (L.w[b] - L.w[a])));
    }
}

// The problem of one pair, from scratch: the y_0 column and the pair's,
// two phases (the artificial basis, then the costs).
void lp_start(const Lifted &L, const Pair &P, DualLP &lp)
{
    const int n = L.n, R = n + 1;
    std::vector<double> cols, costs;
    for (int j = 0; j < n; j++) cols.push_back(0.0);  // y_0 (tau <= 1)
    cols.push_back(1.0);
    costs.push_back(1.0);
    pair_columns(L, P, cols, costs);
    lp.R = R;
    lp.C = (int)costs.size();
    lp.A = cols;  // the artificial basis is the identity: B^-1 M = M
    lp.cost = costs;
    lp.cmax = 0.0;
    for (double c : costs) lp.cmax = std::max(lp.cmax, std::fabs(c));
    lp.Binv.assign((size_t)R * R, 0.0);
    for (int k = 0; k < R; k++) lp.Binv[(size_t)k * R + k] = 1.0;
    lp.rhs.assign(R, 0.0);
    lp.rhs[n] = 1.0;
    lp.basis.resize(R);
    for (int k = 0; k < R; k++) lp.basis[k] = -1 - k;
    // phase 1: minimise the sum of the artificials (multipliers all 1)
    lp.pi.assign(R, 1.0);
    lp.d.resize(lp.C);
    for (int j = 0; j < lp.C; j++) {
        double s = 0.0;
        for (int i = 0; i < R; i++) s += lp.A[(size_t)j * R + i];
        lp.d[j] = -s;
    }
    lp.z = 1.0;
    int rc = lp.run(1e-10);
    if (rc == 3 || lp.z > 1e-9) {
        lp.status = rc == 3 ? 3 : 2;
        return;
    }
    for (int i = 0; i < R; i++) {  // artificials out of the basis where a real column can replace them
        if (lp.basis[i] >= 0) continue;
        for (int j = 0; j < lp.C; j++)
            if (std::fabs(lp.A[(size_t)j * R + i]) > 1e-9) {
                lp.pivot(i, j);
                break;
            }
    }
    // phase 2: the real costs
    lp.pi.assign(R, 0.0);
    lp.z = 0.0;
    for (int i = 0; i < R; i++) {
        const double cb = lp.basis[i] >= 0 ? lp.cost[lp.basis[i]] : 0.0;
        if (cb == 0.0) continue;
        for (int k = 0; k < R; k++) lp.pi[k] += cb * lp.Binv[(size_t)i * R + k];
        lp.z += cb * lp.rhs[i];
    }
    for (int j = 0; j < lp.C; j++) {
        double s = lp.cost[j];
        for (int i = 0; i < R; i++) {
            const double cb = lp.basis[i] >= 0 ? lp.cost[lp.basis[i]] : 0.0;
            s -= cb * lp.A[(size_t)j * R + i];
        }
        lp.d[j] = s;
    }
    rc = lp.run(1e-10 * (1.0 + lp.cmax));
    lp.status = rc;
}

// The parent's problem with the columns of one more pair, continued from the
// parent's basis.
void lp_extend(const Lifted &L, const DualLP &parent, const Pair &P, DualLP &lp)
{
    lp = parent;
    thread_local std::vector<double> cols, costs;
    cols.clear();
    costs.clear();
    pair_columns(L, P, cols, costs);
    const int R = lp.R;
    lp.A.reserve((size_t)(lp.C + costs.size()) * R);
    lp.d.reserve(lp.C + costs.size());
    lp.cost.reserve(lp.C + costs.size());
    for (size_t c = 0; c < costs.size(); c++) lp.add_column(&cols[c * R], costs[c]);
    // an artificial left in the basis (at 0) holds a row no parent column
    // touched; a new column that touches it replaces it (a degenerate pivot:
    // the basis stays feasible), before the simplex may move that row
    for (int i = 0; i < R; i++) {
        if (lp.basis[i] >= 0) continue;
        for (int j = 0; j < lp.C; j++)
            if (std::fabs(lp.A[(size_t)j * R + i]) > 1e-9) {
                lp.pivot(i, j);
                break;
            }
    }
    // the node is pruned once its objective is below the threshold of
    // lp_feasible: the simplex keeps the basis feasible and the objective
    // only falls, so the minimum lies below it too
    lp.status = lp.run(1e-10 * (1.0 + lp.cmax), -1e-7 * (1.0 + L.wmax));
}

// Feasibility from a solved problem (as feasible()).
bool lp_feasible(const Lifted &L, const DualLP &lp)
{
    if (lp.status == 1 || lp.status == 2 || lp.status == 4) return false;
    if (lp.status != 0) return true;
    return lp.z > -1e-7 * (1.0 + L.wmax);
}

// ------------------------------------------------------------------ exact arithmetic

bool mul_ok(i128 a, i128 b, i128 *out) { return !__builtin_mul_overflow(a, b, out); }
bool add_ok(i128 a, i128 b, i128 *out) { return !__builtin_add_overflow(a, b, out); }

// Determinant by fraction-free (Bareiss) elimination; false on overflow.
bool det_exact(int n, std::vector<i128> M, i128 *out)
{
    i128 prev = 1;
    int sign = 1;
    for (int k = 0; k < n - 1; k++) {
        if (M[(size_t)k * n + k] == 0) {
            int p = -1;
            for (int i = k + 1; i < n; i++)
                if (M[(size_t)i * n + k] != 0) {
                    p = i;
                    break;
                }
            if (p < 0) {
                *out = 0;
                return true;
            }
            for (int j = 0; j < n; j++) std::swap(M[(size_t)k * n + j], M[(size_t)p * n + j]);
            sign = -sign;
        }
        for (int i = k + 1; i < n; i++)
            for (int j = k + 1; j < n; j++) {
                i128 u, v;
                if (!mul_ok(M[(size_t)i * n + j], M[(size_t)k * n + k], &u)) return false;
                if (!mul_ok(M[(size_t)i * n + k], M[(size_t)k * n + j], &v)) return false;
                M[(size_t)i * n + j] = (u - v) / prev;
            }
        prev = M[(size_t)k * n + k];
    }
    *out = sign * M[(size_t)(n - 1) * n + n - 1];
    return true;
}

// Exact data of a complete choice: det D and x = det * v (Cramer), then the
// scaled levels E_t = det * (<A_t, v> + w_t - beta_i) * sign(det) >= 0 of
// every term.  Returns 1 for a fine mixed cell, 0 for no cell, -1 on a tie
// (a choice that is otherwise a cell with a third point on its lower facet),
// -2 on overflow.
int exact_cell(const Lifted &L, const Pair *P, i128 *det_out, std::vector<i128> *E)
{
    const int n = L.n;
    std::vector<i128> D((size_t)n * n);
    std::vector<i128> r(n);
    for (int i = 0; i < n; i++) {
        for (int j = 0; j < n; j++) D[(size_t)i * n + j] = L.at(P[i].b, j) - L.at(P[i].a, j);
        r[i] = L.w[P[i].a] - L.w[P[i].b];
    }
    i128 det = 0;
    if (!det_exact(n, D, &det)) return -2;
    if (det == 0) return 0;
    std::vector<i128> x(n);
    for (int j = 0; j < n; j++) {
        std::vector<i128> Dj = D;
        for (int i = 0; i < n; i++) Dj[(size_t)i * n + j] = r[i];
        if (!det_exact(n, Dj, &x[j])) return -2;
    }
    const i128 sgn = det < 0 ? -1 : 1;
    if (E) E->assign(L.A.size() / n, 0);
    // a point below the pair's level rules the choice out; a tie matters
    // only for a choice that is otherwise a cell
    int result = 1;
    bool tie = false;
    auto level = [&](int t, i128 *out) -> bool {
        i128 s = 0, u;
        for (int j = 0; j < n; j++)
            if (!mul_ok((i128)L.at(t, j), x[j], &u) || !add_ok(s, u, &s)) return false;
        if (!mul_ok((i128)L.w[t], det, &u) || !add_ok(s, u, &s)) return false;
        *out = s;
        return true;
    };
    for (int i = 0; i < n; i++) {
        i128 base;
        if (!level(P[i].a, &base)) return -2;
        for (int c = L.off[i]; c < L.off[i] + L.m[i]; c++) {
            i128 val, diff;
            if (!level(c, &val)) return -2;
            if (__builtin_sub_overflow(val, base, &diff)) return -2;
            diff *= sgn;
            if (E) (*E)[c] = diff;
            if (c == P[i].a || c == P[i].b) continue;  // equal level: v solves the pair's equation
            if (diff == 0) tie = true;
            if (diff < 0) result = 0;
        }
        if (result == 0 && !E) return 0;
    }
    *det_out = det;
    if (result == 1 && tie) return -1;
    return result;
}

int load(int n, const int32_t *tpe, const uint8_t *exps, const int32_t *lift, Lifted *L)
{
    if (n < 1 || n > PHC_MAX_VARS) return set_error(PHC_EINVAL, "mixed cells: n outside 1..PHC_MAX_VARS");
    if (!tpe || !exps || !lift) return set_error(PHC_EINVAL, "mixed cells: NULL list");
    L->n = n;
    int T = 0;
    for (int i = 0; i < n; i++) {
        if (tpe[i] < 1 || tpe[i] > 4096) return set_error(PHC_EINVAL, "mixed cells: terms per equation outside 1..4096");
        L->off.push_back(T);
        L->m.push_back(tpe[i]);
        T += tpe[i];
    }
    L->A.resize((size_t)T * n);
    L->w.resize(T);
    for (int t = 0; t < T; t++) {
        for (int j = 0; j < n; j++) L->A[(size_t)t * n + j] = exps[(size_t)t * n + j];
        if (lift[t] < 0 || lift[t] > (1 << 20))
            return set_error(PHC_EINVAL, "mixed cells: lifting values must lie in 0..2^20");
        L->w[t] = lift[t];
        L->wmax = std::max(L->wmax, (double)lift[t]);
    }
    for (int i = 0; i < n; i++)
        for (int a = L->off[i]; a < L->off[i] + L->m[i]; a++)
            for (int b = a + 1; b < L->off[i] + L->m[i]; b++)
                if (std::memcmp(&L->A[(size_t)a * n], &L->A[(size_t)b * n], n * sizeof(int64_t)) == 0)
                    return set_error(PHC_EINVAL, "mixed cells: an equation lists a monomial twice");
    return PHC_OK;
}

bool gcd_ext(int64_t a, int64_t b, int64_t *g, int64_t *s, int64_t *t)
{
    // s a + t b = g = gcd(a, b) >= 0
    int64_t r0 = a, r1 = b, s0 = 1, s1 = 0, t0 = 0, t1 = 1;
    while (r1 != 0) {
        const int64_t q = r0 / r1;
        int64_t u, v;
        if (__builtin_mul_overflow(q, r1, &u) || __builtin_sub_overflow(r0, u, &v)) return false;
        r0 = r1;
        r1 = v;
        if (__builtin_mul_overflow(q, s1, &u) || __builtin_sub_overflow(s0, u, &v)) return false;
        s0 = s1;
        s1 = v;
        if (__builtin_mul_overflow(q, t1, &u) || __builtin_sub_overflow(t0, u, &v)) return false;
        t0 = t1;
        t1 = v;
    }
    if (r0 < 0) {
        r0 = -r0;
        s0 = -s0;
        t0 = -t0;
    }
    *g = r0;
    *s = s0;
    *t = t0;
    return true;
}

}  // namespace

namespace {

// Joins the threads of a pool on every way out of a scope (an exception
// included), after telling them to stop.
struct PoolGuard {
    std::vector<std::thread> &pool;
    std::atomic<bool> *stop;
    ~PoolGuard()
    {
        if (stop) *stop = true;
        for (auto &th : pool)
            if (th.joinable()) th.join();
    }
};

// Runs fn(k) for k = 0 .. count-1 on the host threads (each k once); false
// when an fn threw (out of host memory).
bool parallel_for(int64_t count, int threads, const std::function<void(int64_t)> &fn)
{
    std::atomic<int64_t> next(0);
    std::atomic<bool> failed(false);
    auto body = [&]() {
        for (int64_t k = next++; k < count && !failed; k = next++) {
            try {
                fn(k);
            } catch (...) {
                failed = true;
            }
        }
    };
    std::vector<std::thread> pool;
    {
        PoolGuard guard{pool, nullptr};
        for (int t = 1; t < threads; t++) pool.emplace_back(body);
        body();
    }
    return !failed;
}

// The host threads of the search: PHC_HOST_THREADS from the environment
// when set (1..64), else the hardware's.
int host_threads()
{
    long h = 0;
    if (const char *e = std::getenv("PHC_HOST_THREADS")) h = std::strtol(e, nullptr, 10);
    if (h < 1) h = (long)std::thread::hardware_concurrency();
    if (h < 1) h = 1;
    if (h > 64) h = 64;
    return (int)h;
}

// The edges related to every chosen edge, and the equation the search takes
// next: of the equations not chosen yet, the one with the fewest such edges
// (the first on ties), so that dead ends show early; -1 when some equation
// has none left (no cell below the chosen edges).
struct Picker {
    int n = 0, words = 0;
    const std::vector<int> *eoff = nullptr, *eq_of = nullptr;
    const std::vector<uint64_t> *rel = nullptr;
    int pick(const int *ids, int d, uint64_t *cand) const
    {
        const int NE = (*eoff)[n];
        for (int w = 0; w < words; w++) cand[w] = ~0ull;
        if (NE % 64) cand[words - 1] = (1ull << (NE % 64)) - 1ull;
        unsigned used = 0;
        for (int k = 0; k < d; k++) {
            const uint64_t *row = &(*rel)[(size_t)ids[k] * words];
            for (int w = 0; w < words; w++) cand[w] &= row[w];
            used |= 1u << (*eq_of)[ids[k]];
        }
        int best = -1, best_count = 0;
        for (int i = 0; i < n; i++) {
            if (used & (1u << i)) continue;
            int count = 0;
            for (int ge = (*eoff)[i]; ge < (*eoff)[i + 1]; ge++) count += (int)((cand[ge / 64] >> (ge % 64)) & 1ull);
            if (count == 0) return -1;
            if (best < 0 || count < best_count) {
                best = i;
                best_count = count;
            }
        }
        return best;
    }
};

// Depth-first search below a fixed prefix of edges; the cells of one task.
struct Walker {
    const Lifted &L;
    const std::vector<std::vector<Pair>> &edges;
    const std::vector<int> &eoff, &eq_of;
    const Picker &picker;
    int words;
    std::vector<Pair> chosen, sorted;
    std::vector<int> chosen_id;
    std::vector<uint64_t> cand;   // one candidate mask per depth
    std::vector<DualLP> lps;      // the problem of chosen[0..d] per depth d
    std::vector<int32_t> cells;   // 2n term indices per cell
    std::vector<int64_t> volumes;
    int status = PHC_OK;          // error messages are set on the calling thread
    const char *message = "";

    Walker(const Lifted &l, const std::vector<std::vector<Pair>> &e, const std::vector<int> &eo,
           const std::vector<int> &eq, const Picker &p, int w)
        : L(l), edges(e), eoff(eo), eq_of(eq), picker(p), words(w), chosen(l.n), sorted(l.n), chosen_id(l.n),
          cand((size_t)l.n * w), lps(l.n)
    {
    }
    // solves the problem of chosen[0..d] (from depth d - 1's when that one
    // was solved to the end); true when it is feasible
    bool solve(int d)
    {
        if (d == 0 || lps[d - 1].status != 0) {
            lp_start(L, chosen[0], lps[0]);
            for (int k = 1; k <= d; k++) lp_extend(L, lps[k - 1], chosen[k], lps[k]);
        } else {
            lp_extend(L, lps[d - 1], chosen[d], lps[d]);
        }
        return lp_feasible(L, lps[d]);
    }
    const Pair &edge(int ge) const { return edges[eq_of[ge]][ge - eoff[eq_of[ge]]]; }
    // chosen[0..d] is set and pairwise related
    void visit(int d)
    {
        const int n = L.n;
        if (d + 1 < n) {
            const bool ok = solve(d);
            if (d >= 1 && !ok) return;
            walk(d + 1);
            return;
        }
        for (int k = 0; k < n; k++) sorted[chosen[k].eq] = chosen[k];
        i128 det = 0;
        const int ex = exact_cell(L, sorted.data(), &det, nullptr);
        if (ex == -1) {
            status = PHC_EINVAL;
            message = "mixed cells: lifting not in general position (a third point on a cell's lower facet); "
                      "draw another lifting";
            return;
        }
        if (ex == -2) {
            status = PHC_EUNSUPPORTED;
            message = "mixed cells: exact arithmetic overflows 128 bits";
            return;
        }
        if (ex == 0) return;
        const i128 vol = det < 0 ? -det : det;
        if (vol > (i128)INT64_MAX) {
            status = PHC_EUNSUPPORTED;
            message = "mixed cells: cell volume above 2^63";
            return;
        }
        for (int k = 0; k < n; k++) {
            cells.push_back(sorted[k].a);
            cells.push_back(sorted[k].b);
        }
        volumes.push_back((int64_t)vol);
    }
    void walk(int d)
    {
        uint64_t *c = &cand[(size_t)d * words];
        const int i = picker.pick(chosen_id.data(), d, c);
        if (i < 0) return;
        for (int ge = eoff[i]; ge < eoff[i + 1] && !status; ge++) {
            if (!((c[ge / 64] >> (ge % 64)) & 1ull)) continue;
            chosen[d] = edge(ge);
            chosen_id[d] = ge;
            visit(d);
        }
    }
};

}  // namespace

// The search is split into tasks, one per choice of its first edges, run on
// the host threads; every task keeps its
// cells, and the tasks' cells are emitted in task order from the calling
// thread as the tasks finish -- the order, and so the cells' order, of the
// sequential search.
int enumerate_mixed_cells(int n, const int32_t *tpe, const uint8_t *exps, const int32_t *lift,
                          const std::function<int(const int32_t *pairs, int64_t volume)> &emit)
{
    Lifted L;
    int rc = load(n, tpe, exps, lift, &L);
    if (rc) return rc;
    const int threads = host_threads();
    // (1) lower edges of every lifted support on its own
    std::vector<Pair> all;
    for (int i = 0; i < n; i++)
        for (int a = L.off[i]; a < L.off[i] + L.m[i]; a++)
            for (int b = a + 1; b < L.off[i] + L.m[i]; b++) all.push_back(Pair{i, a, b});
    std::vector<char> lower(all.size(), 0);
    if (!parallel_for((int64_t)all.size(), threads, [&](int64_t k) { lower[k] = feasible(L, &all[k], 1); }))
        return set_error(PHC_ENOMEM, "mixed cells: host allocation failed");
    std::vector<std::vector<Pair>> edges(n);
    for (size_t k = 0; k < all.size(); k++)
        if (lower[k]) edges[all[k].eq].push_back(all[k]);
    for (int i = 0; i < n; i++)
        if (edges[i].empty()) return PHC_OK;  // a support of one point: no cell, mixed volume 0
    // (2) relation table: edge e of one equation and f of a later one, feasible
    // together (rows computed in parallel, then mirrored)
    std::vector<int> eoff(n + 1, 0);
    for (int i = 0; i < n; i++) eoff[i + 1] = eoff[i] + (int)edges[i].size();
    const int NE = eoff[n];
    const int words = (NE + 63) / 64;
    std::vector<uint64_t> rel((size_t)NE * words, 0);
    std::vector<int> eq_of(NE);
    for (int i = 0; i < n; i++)
        for (int e = eoff[i]; e < eoff[i + 1]; e++) eq_of[e] = i;
    const bool rel_ok = parallel_for(NE, threads, [&](int64_t ge) {
        const int i = eq_of[ge];
        const Pair &pe = edges[i][ge - eoff[i]];
        for (int gf = eoff[i + 1]; gf < NE; gf++) {
            const int j = eq_of[gf];
            const Pair two[2] = {pe, edges[j][gf - eoff[j]]};
            if (feasible(L, two, 2)) rel[(size_t)ge * words + gf / 64] |= 1ull << (gf % 64);
        }
    });
    if (!rel_ok) return set_error(PHC_ENOMEM, "mixed cells: host allocation failed");
    for (int ge = 0; ge < NE; ge++)
        for (int gf = eoff[eq_of[ge] + 1]; gf < NE; gf++)
            if ((rel[(size_t)ge * words + gf / 64] >> (gf % 64)) & 1ull) rel[(size_t)gf * words + ge / 64] |= 1ull << (ge % 64);
    // (3) tasks: the choices of the first P edges the search makes (its
    // ordering by fewest related edges, without the linear programs), P the
    // smallest depth that gives 32 tasks per thread (or n), in the order of
    // the sequential search
    Picker picker;
    picker.n = n;
    picker.words = words;
    picker.eoff = &eoff;
    picker.eq_of = &eq_of;
    picker.rel = &rel;
    std::vector<std::vector<int>> prefixes(1);
    int P = 0;
    std::vector<uint64_t> cmask(words);
    while (P < n && prefixes.size() < (size_t)32 * threads) {
        std::vector<std::vector<int>> longer;
        for (const auto &pre : prefixes) {
            const int i = picker.pick(pre.data(), P, cmask.data());
            if (i < 0) continue;
            for (int ge = eoff[i]; ge < eoff[i + 1]; ge++)
                if ((cmask[ge / 64] >> (ge % 64)) & 1ull) {
                    longer.push_back(pre);
                    longer.back().push_back(ge);
                }
        }
        prefixes.swap(longer);
        P++;
    }
    const int64_t NT = P == 0 ? 0 : (int64_t)prefixes.size();
    std::vector<std::unique_ptr<Walker>> done(NT);
    std::vector<char> finished(NT, 0);  // 1 done, 2 out of host memory
    std::mutex mu;
    std::condition_variable cv;
    std::atomic<int64_t> next(0);
    std::atomic<bool> stop(false);
    auto worker = [&]() {
        for (int64_t k = next++; k < NT && !stop; k = next++) {
            std::unique_ptr<Walker> w;
            char how = 1;
            try {
                w.reset(new Walker(L, edges, eoff, eq_of, picker, words));
                const auto &pre = prefixes[k];
                for (int d = 0; d < P; d++) {
                    w->chosen[d] = w->edge(pre[d]);
                    w->chosen_id[d] = pre[d];
                }
                // the tests the sequential search makes on the way to depth P - 1
                bool ok = true;
                for (int d = 0; d + 1 < P && ok; d++) ok = w->solve(d) || d == 0;
                if (ok) w->visit(P - 1);
            } catch (...) {
                how = 2;
            }
            std::lock_guard<std::mutex> lock(mu);
            done[k] = std::move(w);
            finished[k] = how;
            cv.notify_all();
        }
    };
    std::vector<std::thread> pool;
    int status = PHC_OK;
    {
        PoolGuard guard{pool, &stop};
        for (int t = 0; t < threads; t++) pool.emplace_back(worker);
        for (int64_t k = 0; k < NT && !status; k++) {
            {
                std::unique_lock<std::mutex> lock(mu);
                cv.wait(lock, [&] { return finished[k] != 0; });
            }
            if (finished[k] == 2) {
                status = set_error(PHC_ENOMEM, "mixed cells: host allocation failed");
                break;
            }
            const Walker &w = *done[k];
            if (w.status) status = set_error(w.status, w.message);
            for (size_t c = 0; c < w.volumes.size() && !status; c++) status = emit(&w.cells[c * 2 * n], w.volumes[c]);
            done[k].reset();
        }
    }
    return status;
}

int cell_tracking_data(int n, const int32_t *tpe, const uint8_t *exps, const int32_t *lift, const int32_t *pairs,
                       double *powers, int64_t *H, int64_t *U, int64_t *volume)
{
    Lifted L;
    int rc = load(n, tpe, exps, lift, &L);
    if (rc) return rc;
    std::vector<Pair> P(n);
    for (int i = 0; i < n; i++) {
        const int a = pairs[2 * i], b = pairs[2 * i + 1];
        if (a < L.off[i] || b < L.off[i] || a >= L.off[i] + L.m[i] || b >= L.off[i] + L.m[i] || a == b)
            return set_error(PHC_EINVAL, "cell: a pair does not name two terms of its equation");
        P[i] = Pair{i, std::min(a, b), std::max(a, b)};
    }
    i128 det = 0;
    std::vector<i128> E;
    const int ex = exact_cell(L, P.data(), &det, &E);
    if (ex == -2) return set_error(PHC_EUNSUPPORTED, "cell: exact arithmetic overflows 128 bits");
    if (ex == -1) return set_error(PHC_EINVAL, "cell: lifting not in general position");
    if (ex == 0) return set_error(PHC_EINVAL, "cell: the pairs are not a fine mixed cell of this lifting");
    // powers: E_t / min positive E (0 on the cell's terms)
    i128 emin = 0;
    for (size_t t = 0; t < E.size(); t++)
        if (E[t] > 0 && (emin == 0 || E[t] < emin)) emin = E[t];
    for (size_t t = 0; t < E.size(); t++) powers[t] = E[t] == 0 ? 0.0 : (double)E[t] / (double)emin;
    // Hermite form: U D = H upper triangular with a positive diagonal, U
    // unimodular (row operations of determinant 1 built from extended gcds)
    std::vector<int64_t> Hm((size_t)n * n), Um((size_t)n * n, 0);
    for (int i = 0; i < n; i++) {
        for (int j = 0; j < n; j++) Hm[(size_t)i * n + j] = L.at(P[i].b, j) - L.at(P[i].a, j);
        Um[(size_t)i * n + i] = 1;
    }
    auto combine = [&](std::vector<int64_t> &M, int k, int i, int64_t s, int64_t t, int64_t p, int64_t q) -> bool {
        // row k := s row_k + t row_i, row i := p row_k + q row_i
        for (int j = 0; j < n; j++) {
            const int64_t rk = M[(size_t)k * n + j], ri = M[(size_t)i * n + j];
            int64_t u, v, x, y;
            if (__builtin_mul_overflow(s, rk, &u) || __builtin_mul_overflow(t, ri, &v) || __builtin_add_overflow(u, v, &x))
                return false;
            if (__builtin_mul_overflow(p, rk, &u) || __builtin_mul_overflow(q, ri, &v) || __builtin_add_overflow(u, v, &y))
                return false;
            M[(size_t)k * n + j] = x;
            M[(size_t)i * n + j] = y;
        }
        return true;
    };
    for (int k = 0; k < n; k++) {
        for (int i = k + 1; i < n; i++) {
            const int64_t a = Hm[(size_t)k * n + k], b = Hm[(size_t)i * n + k];
            if (b == 0) continue;
            int64_t g, s, t;
            if (!gcd_ext(a, b, &g, &s, &t)) return set_error(PHC_EUNSUPPORTED, "cell: Hermite form overflows");
            // [s t; -b/g a/g] has determinant (s a + t b) / g = 1
            const int64_t p = -(b / g), q = a / g;
            if (!combine(Hm, k, i, s, t, p, q) || !combine(Um, k, i, s, t, p, q))
                return set_error(PHC_EUNSUPPORTED, "cell: Hermite form overflows");
        }
        if (Hm[(size_t)k * n + k] == 0) return set_error(PHC_EINVAL, "cell: singular exponent matrix");
        if (Hm[(size_t)k * n + k] < 0)
            for (int j = 0; j < n; j++) {
                Hm[(size_t)k * n + j] = -Hm[(size_t)k * n + j];
                Um[(size_t)k * n + j] = -Um[(size_t)k * n + j];
            }
    }
    int64_t prod = 1;
    for (int k = 0; k < n; k++)
        if (__builtin_mul_overflow(prod, Hm[(size_t)k * n + k], &prod))
            return set_error(PHC_EUNSUPPORTED, "cell: volume overflows");
    const i128 vol = det < 0 ? -det : det;
    if ((i128)prod != vol) return set_error(PHC_EINVAL, "internal: Hermite diagonal does not multiply to the volume");
    std::memcpy(H, Hm.data(), Hm.size() * sizeof(int64_t));
    std::memcpy(U, Um.data(), Um.size() * sizeof(int64_t));
    *volume = (int64_t)vol;
    return PHC_OK;
}

}  // namespace phc

static int mixed_cells_impl(int n, const int32_t *terms_per_eq, const uint8_t *exps, const int32_t *lift,
                            int64_t max_cells, int32_t *cells_out, int64_t *volumes_out, int64_t *n_cells_out,
                            int64_t *mixed_volume_out)
{
    if (!n_cells_out) return phc::set_error(PHC_EINVAL, "phc_mixed_cells: n_cells_out is NULL");
    if (max_cells < 0) return phc::set_error(PHC_EINVAL, "phc_mixed_cells: max_cells < 0");
    if (max_cells > 0 && !cells_out) return phc::set_error(PHC_EINVAL, "phc_mixed_cells: cells_out is NULL");
    int64_t count = 0, mv = 0;
    const int rc = phc::enumerate_mixed_cells(n, terms_per_eq, exps, lift, [&](const int32_t *p, int64_t vol) -> int {
        if (count < max_cells) {
            std::memcpy(cells_out + (size_t)count * 2 * n, p, 2 * (size_t)n * sizeof(int32_t));
            if (volumes_out) volumes_out[count] = vol;
        }
        count++;
        if (__builtin_add_overflow(mv, vol, &mv))
            return phc::set_error(PHC_EUNSUPPORTED, "phc_mixed_cells: mixed volume above 2^63");
        return PHC_OK;
    });
    if (rc) return rc;
    *n_cells_out = count;
    if (mixed_volume_out) *mixed_volume_out = mv;
    return PHC_OK;
}

extern "C" int phc_mixed_cells(int n, const int32_t *terms_per_eq, const uint8_t *exps, const int32_t *lift,
                               int64_t max_cells, int32_t *cells_out, int64_t *volumes_out, int64_t *n_cells_out,
                               int64_t *mixed_volume_out)
{
    try {
        return mixed_cells_impl(n, terms_per_eq, exps, lift, max_cells, cells_out, volumes_out, n_cells_out,
                                mixed_volume_out);
    } catch (...) {
        return phc::set_error(PHC_ENOMEM, "phc_mixed_cells: host allocation failed");
    }
}
