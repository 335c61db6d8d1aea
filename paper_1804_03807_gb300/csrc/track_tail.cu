// track_tail.cu -- the tail kernels: G threads per path.
//
// When most lanes of a tracking launch have run out of paths, the remaining
// paths leave the one-thread-per-path kernel at the start of a step (see the
// hand-off in track_impl.cuh) and continue here with a group of G lanes per
// path (tail_path in tail_impl.cuh), so that a long path no longer runs at the
// speed of one thread that shares an FP64 pipe with a mostly empty warp.
#include "tail_impl.cuh"

namespace phc {

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
        const size_t cs = (size_t)hd.sys * tb.n_terms;
        tail_path<N, G>(hd, tb, plan, LinearCoef{tb.c0 + cs, tb.c1 + cs}, base, L.o, r, gmask,
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
        tail_path<N, G>(hd, tb, plan, LinearCoef{tb.c0, tb.c1}, base, L.o, r, 0xffffffffu,
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
            tail_path<N, G>(*cur, tb, stage ? plan2 : plan1, LinearCoef{tb.c0, tb.c1}, base, o, r, FULL,
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
