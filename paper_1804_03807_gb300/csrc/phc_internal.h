// Internal declarations shared by the host API (phc_api.cpp) and the CUDA
// kernels (track.cu, refine.cu).  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <functional>
#include <cuda_runtime.h>

#include "../../include/phc.h"

namespace phc {

// One term of a homotopy H(x,t) = sum_terms (c0 + t c1) x^a, stored as the
// support of x^a: k variables vars[off..off+k) with exponents exps[off..).
// Every homotopy the library tracks has coefficients linear in t:
//   total degree  f terms (0, c);  x_i^{d_i}: (gamma, -gamma);  -1: (-gamma, gamma)
//   cascade       E_k terms (c, 0);  hyperplane k without z_k: (c, -c)
struct TermRec {
    uint8_t eq;     // equation (row of H)
    uint8_t k;      // support size
    uint8_t flags;  // bit 0: some exponent > 1
    uint8_t pad;
    uint16_t off;   // offset into vars / exps
    uint16_t pad2;
};
static_assert(sizeof(TermRec) == 8, "TermRec layout");

enum : uint8_t { TERM_POWERS = 1 };

// Device tables of one homotopy (global memory; staged into shared memory
// by the kernels).
// A batch of n_sys homotopies shares terms/vars/exps; system s has the
// coefficients c0[s * n_terms + q], c1[s * n_terms + q].  Terms are grouped
// by equation in ascending order (upload_table checks it; the tail kernel
// relies on it).
struct DevTables {
    int n;        // unknowns = equations
    int n_terms;  // terms
    int n_ve;     // entries of vars / exps
    int n_sys;    // systems sharing the structure
    int f32;      // the single precision copies are staged and used (FP32 interior); the
                  // launchers clear it for double precision work
    int coef_smem;  // stage the coefficients into shared memory (when within
                    // COEF_SMEM_LIMIT); the tail launcher clears it when its
                    // term store would not fit otherwise
    const TermRec *terms;
    const uint8_t *vars;
    const uint8_t *exps;
    const double2 *c0;
    const double2 *c1;
    const float2 *c0f;  // single precision copies (FP32 interior)
    const float2 *c1f;
};

// Bytes of coefficients per term and system: c0, c1 in double and, with
// f32, c0, c1 in float.
__host__ __device__ inline size_t coef_bytes(bool f32) { return f32 ? 2 * 16 + 2 * 8 : 2 * 16; }
// Coefficients of all systems are staged into shared memory up to this size;
// larger batches read them through L1.
constexpr size_t COEF_SMEM_LIMIT = 48 * 1024;

__host__ __device__ inline bool coefs_in_smem(const DevTables &t)
{
    return t.coef_smem && (size_t)t.n_terms * (size_t)t.n_sys * coef_bytes(t.f32) <= COEF_SMEM_LIMIT;
}

// Bytes the staged copy of a table takes in shared memory (16-byte aligned).
__host__ __device__ inline size_t table_smem_bytes(const DevTables &t)
{
    size_t b = (size_t)t.n_terms * sizeof(TermRec) + 2 * (size_t)t.n_ve;
    b = (b + 15) & ~(size_t)15;
    if (coefs_in_smem(t)) b += (size_t)t.n_terms * (size_t)t.n_sys * coef_bytes(t.f32);
    return b;
}

// Per-thread shared memory: the evaluation point xe, the right-hand side R,
// prefix products P (N slots each), with f32 the single precision point X
// (N slots), the Jacobian J (N*N slots) and, for classification, the scales
// S (N slots); one slot is a complex double (single precision values use its
// first half).  Without X a 160-thread block of the 7-unknown tracker grows
// to 192 threads.
// With localp the prefix products live in the thread's local memory (L1)
// instead of shared memory: N fewer slots, which lets the single-homotopy
// tracker hold more threads per block for the numbers of unknowns in
// PHC_LOCALP_MASK (bit N set).  The default takes N = 7, 8 and 11, where the
// block grows (N = 11: from 64 to 96 threads, 2 to 3 of the 4 SM partitions
// busy; the cyclic 9 D=2 top stage went from 12.57 to 8.54 s; N = 7, 8: from
// 160 to 192 and from 128 to 160 threads, 2 % faster); for the other N the
// block size is the same either way (or already at 256 threads).
__host__ __device__ inline size_t thread_smem_bytes(int n, bool scale = false, bool f32 = true, bool localp = false)
{
    return (size_t)(n * n + 3 * n - (localp ? n : 0) + (f32 ? n : 0) + (scale ? n : 0)) * sizeof(double2);
}
#ifndef PHC_LOCALP_MASK
#define PHC_LOCALP_MASK ((1u << 7) | (1u << 8) | (1u << 11))
#endif
__host__ __device__ constexpr bool localp_of(int n) { return ((PHC_LOCALP_MASK) >> n) & 1u; }
// The same for the pipelined tracker (top stage and cascade stage in one
// launch), whose threads also keep the classification scales: N = 7, 8 and 9
// gain a warp per block (160 -> 192, 128 -> 160, 96 -> 128 threads).
#ifndef PHC_LOCALP_PIPE_MASK
#define PHC_LOCALP_PIPE_MASK ((1u << 7) | (1u << 8) | (1u << 9))
#endif
__host__ __device__ constexpr bool localp_pipe_of(int n) { return ((PHC_LOCALP_PIPE_MASK) >> n) & 1u; }

// One system of a multi-system launch (systems of different structure and
// equal number of unknowns tracked in one kernel).
struct SysDesc {
    DevTables tab;
    const int32_t *deg;
    const int32_t *root_off;
    const double2 *roots;
    int64_t n_paths;
    double2 *x_out;           // SoA [n][n_paths]
    int8_t *cls_out;          // [n_paths]
    phc_path_stats *stats;    // [n_paths]
};

// The state of a path at the start of a step, handed from the tracker to
// a tail kernel when most lanes have run out of paths.
struct Handoff {
    double2 x0[PHC_MAX_VARS];
    double t, h, next_s, nx0, r0, r1, r2, r3, r4;
    int64_t q;
    int32_t sys, streak, steps, since_ck, nck, n_acc, n_rej, n_newt, n_solve, n_f32;
    int32_t stage;  // pipelined launch: 0 top homotopy, 1 cascade stage
};

struct TrackLaunch {
    DevTables tab;
    // starts: mode 0 = total-degree roots of unity, mode 1 = explicit SoA
    int start_mode;
    const int32_t *deg;       // [n]
    const int32_t *root_off;  // [n]
    const double2 *roots;     // [sum deg]
    const double2 *starts;    // SoA [n][n_paths] (modes 1 and 2)
    const int8_t *sel_cls;    // mode 2: track entry q only if sel_cls[q] is regular
    const uint8_t *sel_sz;    //         and sel_sz[q] == 0 (NULL: test the last slack of starts)
    int64_t first;
    int64_t n_paths;
    int64_t paths_per_system; // global path p belongs to system p / paths_per_system
    int64_t starts_per_system;  // modes 1 and 2: entry q belongs to system q / starts_per_system (0: system 0)
    double2 *x_out;           // SoA [n][n_paths]
    phc_path_stats *stats;    // [n_paths]
    unsigned long long *qhead;
    phc_opts o;
    // pipeline: the cascade stage of tab2 continues every top endpoint that
    // is regular with a nonzero last slack, in the same lane
    DevTables tab2;
    int8_t *cls_out;          // [n_paths] top-stage classes
    double2 *x_out2;          // SoA [n - 1][n_paths]
    int8_t *cls_out2;         // [n_paths], -1 when the path was not continued
    uint8_t *slack_zero2;     // [n_paths]
    phc_path_stats *stats2;   // [n_paths]
    int has_next_slack;       // the stage's endpoints keep a slack z_{k-1}
    // multi-system launch: every warp tracks one system at a time
    const SysDesc *multi;     // [n_multi]
    unsigned long long *multi_q;   // [n_multi] path counters
    const int64_t *multi_prefix;   // [n_multi + 1] prefix sums of path counts
    int n_multi;
    int warp_table_bytes;     // shared memory per warp for one system's table
    // tail hand-off (mode 0, double precision): when idle_n reaches drain_at,
    // lanes that start a new step save their path to handoff[] and leave
    Handoff *handoff;
    unsigned long long *handoff_n;
    unsigned long long *idle_n;
    unsigned long long *tail_q;
    unsigned long long *tail_units;  // units the tail kernel ran (diagnostic)
    unsigned long long *multi_claimed;  // multi-system: paths claimed over all systems
    unsigned long long drain_at;  // set by the launcher from drain_frac
    double drain_frac;            // fraction of idle lanes that starts the hand-off; 0: never
    int compact;                  // single-homotopy mode: move running paths to the lowest lanes
                                  // of their block once the queue is empty (N >= 4)
    int64_t handoff_cap;          // records the hand-off buffer holds; 0: one per lane.  With a
                                  // cap the hand-off starts no earlier than when at most this many
                                  // lanes still hold a path (each writes one record at most)
};

// Bytes of shared memory one warp needs for a table of T terms and V
// exponent entries (single system, 16-byte aligned).
__host__ __device__ inline size_t warp_table_bytes(int T, int V, bool f32)
{
    size_t b = (size_t)T * sizeof(TermRec) + 2 * (size_t)V;
    b = (b + 15) & ~(size_t)15;
    return b + (size_t)T * coef_bytes(f32);
}

struct ClassifyLaunch {
    DevTables tab;
    int64_t n_paths;
    const double2 *x;         // SoA [n][x_ld] (x_ld 0: n_paths)
    int64_t x_ld;
    phc_path_stats *stats;    // [n_paths] in/out
    int8_t *cls;              // [n_paths] out
    phc_opts o;
};

struct RefineLaunch {
    DevTables tab;
    int64_t n;
    double2 *x_hi;            // SoA [n_var][n]
    double2 *x_lo;            // SoA [n_var][n]
    int8_t *cls;
    phc_path_stats *stats;
    double cond_threshold, cond_max;
    int max_iters;
    phc_opts o;
};

// Launchers (track.cu / refine.cu).  Each returns a cudaError_t.
cudaError_t launch_roots(const int32_t *deg, const int32_t *root_off, double2 *roots, int n, int total,
                         cudaStream_t s);
cudaError_t launch_track(const TrackLaunch &L, int block_threads, int max_blocks, cudaStream_t s);
cudaError_t launch_pipeline(const TrackLaunch &L, int block_threads, int max_blocks, cudaStream_t s);
cudaError_t launch_multi(const TrackLaunch &L, int n, int block_threads, int max_blocks, cudaStream_t s);
// Lanes the tracker launches for L (grid x block), for sizing the hand-off buffer.
int64_t track_lanes(const TrackLaunch &L, int block_threads, int max_blocks);
// The paths handed off by launch_track (L.handoff), L.o.tail_threads threads
// per path; tail_supported: the tail kernel can hold one path of this table.
cudaError_t launch_tail(const TrackLaunch &L, int max_blocks, cudaStream_t s);
bool tail_supported(const DevTables &t);

// Shared memory of the tail kernels (see track_tail.cu): the evaluation plan
// of a table (term slots and orders, each entry's pieces; 16-bit words) ...
inline size_t tail_plan_bytes(int n, int T, int n_ve)
{
    const int E = n * n + n;
    const size_t b = 2 * ((size_t)T + T + (E + 1) + (n_ve + T) + E);
    return (b + 15) & ~(size_t)15;
}
// ... the term store of one path (2k + 1 slots per term with k >= 1, 1 per
// constant) ...
__host__ __device__ inline int tail_store_slots(int T, int n_ve) { return 2 * n_ve + T; }
// ... and a group's slots: xe, R (N each), J (N^2) and the store, which also
// holds the one-lane classification arrays of the multi-system tail.
__host__ __device__ inline int tail_group_slots(int n, int S)
{
    const int cls = n * n + 5 * n;
    return 2 * n + n * n + (S > cls ? S : cls);
}
// Per-warp region of the multi-system tail kernel: the largest table, plan
// and group over the systems of the launch.
struct TailMultiSizes {
    size_t table_cap, plan_cap;
    int group_slots, max_store;
};
// The paths handed off by a multi-system launch (one warp per path).
cudaError_t launch_tail_multi(const TrackLaunch &L, int n, const TailMultiSizes &z, int max_blocks, cudaStream_t s);
bool tail_multi_supported(const TailMultiSizes &z);
// Lanes a multi-system launch of L runs (for sizing its hand-off buffer).
int64_t multi_lanes(const TrackLaunch &L, int n, int block_threads, int max_blocks);
// The paths handed off by a pipelined launch (top stage and cascade stage),
// one warp per path; the lanes such a launch runs; whether the tail fits.
cudaError_t launch_tail_pipe(const TrackLaunch &L, int max_blocks, cudaStream_t s);
int64_t pipe_lanes(const TrackLaunch &L, int block_threads, int max_blocks);
bool tail_pipe_supported(const DevTables &t1, const DevTables &t2);
cudaError_t launch_classify(const ClassifyLaunch &L, cudaStream_t s);
// Total-degree paths of L tracked in complex double double (track_dd.cu):
// double parts to L.x_out, low parts to L.x_out2, records to L.stats.
cudaError_t launch_track_dd(const TrackLaunch &L, int block_threads, int max_blocks, cudaStream_t s);
// Total-degree paths of L tracked in complex quad double (track_qd.cu): the
// four parts of every coordinate to L.x_out, SoA [4][n][n_paths] (part-major),
// records to L.stats.
cudaError_t launch_track_qd(const TrackLaunch &L, int block_threads, int max_blocks, cudaStream_t s);
// The Cauchy endgame of the total-degree paths of L (endgame.cu): estimates
// to L.x_out, records to L.stats, cycle numbers (0: no estimate) to cycle_out.
cudaError_t launch_endgame(const TrackLaunch &L, int32_t *cycle_out, int block_threads, int max_blocks, cudaStream_t s);
cudaError_t launch_refine(const RefineLaunch &L, cudaStream_t s);
// match[j] = 1 when one of the m endpoints x[:, j*m .. j*m+m) (SoA over
// p*m entries, N unknowns) of class PHC_REGULAR or PHC_SINGULAR equals
// points[:, j] (SoA [n_pt][p]) in its first n_pt unknowns and has its other
// unknowns (the slacks) zero, within tol (1 + ||points_j||).
cudaError_t launch_match_points(const double2 *x, const int8_t *cls, int N, int64_t m, int64_t p,
                                const double2 *points, int n_pt, double tol, uint8_t *match, cudaStream_t s);
// Copies the m start points (SoA [N][m]) p times: out SoA [N][p*m].
cudaError_t launch_tile_starts(const double2 *starts, int N, int64_t m, int64_t p, double2 *out, cudaStream_t s);
cudaError_t launch_drop_last(const double2 *x_full, int n_full, int64_t n_paths, double2 *x_out,
                             uint8_t *slack_zero, int has_next_slack, double slack_tol, cudaStream_t s);

// Polyhedral homotopies of one system g (track_poly.cu): tab holds g's terms
// with the coefficients in c1 (c0 = 0); path p belongs to the cell c with
// path_off[c] <= p < path_off[c + 1].
struct PolyLaunch {
    DevTables tab;
    int n_cells;
    const int64_t *path_off;  // [n_cells + 1]
    const double *powers;     // [n_cells][n_terms] power of t per term
    const int64_t *H, *U;     // [n_cells][n][n] Hermite form U D = H
    const int32_t *pairs;     // [n_cells][n][2] the cell's terms per equation
    int64_t first, n_paths;
    double2 *x_out;           // SoA [n][x_ld] (x_ld 0: n_paths)
    int64_t x_ld;
    phc_path_stats *stats;    // [n_paths]
    unsigned long long *qhead;
    phc_opts o;
};
cudaError_t launch_poly_starts(const PolyLaunch &L, cudaStream_t s);
cudaError_t launch_track_poly(const PolyLaunch &L, int block_threads, int max_blocks, cudaStream_t s);

// Fine mixed cells of the supports under an integer lifting (mixed_cells.cpp,
// host): emit(pairs, volume) once per cell as it is found, pairs = the 2n
// global term indices (a_i, b_i), a_i < b_i, per equation; a nonzero return
// of emit stops the enumeration and is returned.
int enumerate_mixed_cells(int n, const int32_t *tpe, const uint8_t *exps, const int32_t *lift,
                          const std::function<int(const int32_t *pairs, int64_t volume)> &emit);
// The polyhedral homotopy data of one cell: powers [T] (power of t per term,
// 0 on the cell's terms, the others divided by the smallest positive one),
// the Hermite form H (upper triangular, positive diagonal) and the unimodular
// U with U D = H (D rows b_i - a_i), both n x n row-major, and the volume.
int cell_tracking_data(int n, const int32_t *tpe, const uint8_t *exps, const int32_t *lift, const int32_t *pairs,
                       double *powers, int64_t *H, int64_t *U, int64_t *volume);

// Threads per block the tracker uses for n unknowns and a table of the given
// size (fills up to the opt-in shared memory of one block).
int track_block_threads(int n, size_t table_bytes, int requested, bool scale = false, bool f32 = true,
                        bool localp = false);

}  // namespace phc
