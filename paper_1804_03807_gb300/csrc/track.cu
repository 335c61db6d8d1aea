// track.cu -- launchers of the single-homotopy tracker, the classification
// and the small kernels (roots of unity, dropping z_k after a cascade stage).
// The kernels themselves are in track_impl.cuh.
#include "track_impl.cuh"

namespace phc {

// ------------------------------------------------------------------ small kernels

__global__ void roots_kernel(const int32_t *deg, const int32_t *root_off, double2 *roots, int n)
{
    const int i = blockIdx.x;
    if (i >= n) return;
    const int d = deg[i];
    for (int k = threadIdx.x; k < d; k += blockDim.x) {
        double s, c;
        sincospi(2.0 * (double)k / (double)d, &s, &c);
        roots[root_off[i] + k] = make_double2(c, s);
    }
}

__global__ void drop_last_kernel(const double2 *x_full, int n_full, int64_t np, double2 *x_out, uint8_t *slack_zero,
                                 int has_next_slack, double slack_tol)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < np; q += (int64_t)gridDim.x * blockDim.x) {
        double nx = 0.0;
        for (int j = 0; j < n_full - 1; j++) {
            const double2 v = x_full[(int64_t)j * np + q];
            x_out[(int64_t)j * np + q] = v;
            const double a = absinf(v);
            if (!(a <= nx)) nx = a;
        }
        uint8_t z = 0;
        if (has_next_slack) z = absinf(x_full[(int64_t)(n_full - 2) * np + q]) <= slack_tol * (1.0 + nx);
        slack_zero[q] = z;
    }
}

// One block per test point j: its m endpoints are compared with the point
// (homotopy membership test, Section 4.1: the point lies on the component
// when it is one of the endpoints of the paths from the witness points).
__global__ void match_points_kernel(const double2 *x, const int8_t *cls, int N, int64_t m, int64_t p,
                                    const double2 *points, int n_pt, double tol, uint8_t *match)
{
    const int64_t j = blockIdx.x;
    if (j >= p) return;
    double np = 0.0;
    for (int l = 0; l < n_pt; l++) {
        const double a = absinf(points[(int64_t)l * p + j]);
        if (!(a <= np)) np = a;
    }
    const double bound = tol * (1.0 + np);
    int hit = 0;
    const int64_t total = p * m;
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
        const int64_t e = j * m + i;
        if (cls[e] != PHC_REGULAR && cls[e] != PHC_SINGULAR) continue;
        bool same = true;
        for (int l = 0; l < N; l++) {
            const double2 v = x[(int64_t)l * total + e];
            const double2 w = l < n_pt ? points[(int64_t)l * p + j] : make_double2(0.0, 0.0);
            const double d = absinf(make_double2(v.x - w.x, v.y - w.y));
            same = same && d <= bound;
        }
        hit |= same ? 1 : 0;
    }
    hit = __syncthreads_or(hit);
    if (threadIdx.x == 0) match[j] = hit ? 1 : 0;
}

__global__ void tile_starts_kernel(const double2 *starts, int N, int64_t m, int64_t p, double2 *out)
{
    const int64_t total = p * m;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % m;
        for (int l = 0; l < N; l++) out[(int64_t)l * total + e] = starts[(int64_t)l * m + i];
    }
}

// ------------------------------------------------------------------ launchers

int g_num_sms = 0, g_smem_optin = 0;

void device_limits()
{
    if (g_num_sms) return;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&g_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
}

int track_block_threads(int n, size_t table_bytes, int requested, bool scale, bool f32, bool localp)
{
    device_limits();
    const size_t per = thread_smem_bytes(n, scale, f32, localp);
    long fit = ((long)g_smem_optin - (long)table_bytes) / (long)per;
    int bt = (int)((fit / 32) * 32);
    if (bt > 256) bt = 256;
    if (requested > 0 && requested < bt) bt = (requested / 32) * 32;
    if (bt < 32) bt = 0;  // does not fit
    return bt;
}

template <int N>
static cudaError_t launch_classify_n(const ClassifyLaunch &L, cudaStream_t s)
{
    const size_t tb = table_smem_bytes(L.tab);
    const int bt = track_block_threads(N, tb, 128, true, false);
    if (bt == 0) return cudaErrorInvalidConfiguration;
    const size_t smem = tb + (size_t)bt * thread_smem_bytes(N, true, false);
    cudaError_t e = cudaFuncSetAttribute(classify_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int64_t grid = (L.n_paths + bt - 1) / bt;
    if (grid > (int64_t)g_num_sms * 8) grid = (int64_t)g_num_sms * 8;
    if (grid < 1) grid = 1;
    classify_kernel<N><<<(unsigned)grid, bt, smem, s>>>(L, tb);
    return cudaGetLastError();
}

cudaError_t launch_track(const TrackLaunch &L, int block_threads, int max_blocks, cudaStream_t s)
{
    device_limits();
    if (L.n_paths <= 0) return cudaSuccess;
    const size_t tb = table_smem_bytes(L.tab) + compact_smem_bytes(256);
    const int bt = track_block_threads(L.tab.n, tb, block_threads, false, L.o.precision == PHC_PREC_FP32_INTERIOR,
                                       localp_of(L.tab.n));
    if (bt == 0) return cudaErrorInvalidConfiguration;
#define PHC_CALL_TRACK(NN) launch_track_n<NN, MODE_SINGLE>(L, bt, max_blocks, L.n_paths, s)
    PHC_DISPATCH_N(L.tab.n, PHC_CALL_TRACK)
#undef PHC_CALL_TRACK
}

int64_t track_lanes(const TrackLaunch &L, int block_threads, int max_blocks)
{
    device_limits();
    const size_t tb = table_smem_bytes(L.tab) + compact_smem_bytes(256);
    const int bt = track_block_threads(L.tab.n, tb, block_threads, false, L.o.precision == PHC_PREC_FP32_INTERIOR,
                                       localp_of(L.tab.n));
    if (bt == 0) return -1;
    switch (L.tab.n) {
    case 1: return lanes_n<1, MODE_SINGLE>(L, bt, max_blocks);
    case 2: return lanes_n<2, MODE_SINGLE>(L, bt, max_blocks);
    case 3: return lanes_n<3, MODE_SINGLE>(L, bt, max_blocks);
    case 4: return lanes_n<4, MODE_SINGLE>(L, bt, max_blocks);
    case 5: return lanes_n<5, MODE_SINGLE>(L, bt, max_blocks);
    case 6: return lanes_n<6, MODE_SINGLE>(L, bt, max_blocks);
    case 7: return lanes_n<7, MODE_SINGLE>(L, bt, max_blocks);
    case 8: return lanes_n<8, MODE_SINGLE>(L, bt, max_blocks);
    case 9: return lanes_n<9, MODE_SINGLE>(L, bt, max_blocks);
    case 10: return lanes_n<10, MODE_SINGLE>(L, bt, max_blocks);
    case 11: return lanes_n<11, MODE_SINGLE>(L, bt, max_blocks);
    case 12: return lanes_n<12, MODE_SINGLE>(L, bt, max_blocks);
    default: return -1;
    }
}

cudaError_t launch_classify(const ClassifyLaunch &L, cudaStream_t s)
{
    device_limits();
    if (L.n_paths <= 0) return cudaSuccess;
#define PHC_CALL_CLS(NN) launch_classify_n<NN>(L, s)
    PHC_DISPATCH_N(L.tab.n, PHC_CALL_CLS)
#undef PHC_CALL_CLS
}

cudaError_t launch_roots(const int32_t *deg, const int32_t *root_off, double2 *roots, int n, int total, cudaStream_t s)
{
    (void)total;
    roots_kernel<<<n, 64, 0, s>>>(deg, root_off, roots, n);
    return cudaGetLastError();
}

cudaError_t launch_match_points(const double2 *x, const int8_t *cls, int N, int64_t m, int64_t p,
                                const double2 *points, int n_pt, double tol, uint8_t *match, cudaStream_t s)
{
    if (p <= 0) return cudaSuccess;
    if (p > 0x7fffffffLL) return cudaErrorInvalidValue;
    match_points_kernel<<<(unsigned)p, 128, 0, s>>>(x, cls, N, m, p, points, n_pt, tol, match);
    return cudaGetLastError();
}

cudaError_t launch_tile_starts(const double2 *starts, int N, int64_t m, int64_t p, double2 *out, cudaStream_t s)
{
    device_limits();
    if (p <= 0 || m <= 0) return cudaSuccess;
    int64_t grid = (p * m + 255) / 256;
    if (grid > (int64_t)g_num_sms * 16) grid = (int64_t)g_num_sms * 16;
    tile_starts_kernel<<<(unsigned)grid, 256, 0, s>>>(starts, N, m, p, out);
    return cudaGetLastError();
}

cudaError_t launch_drop_last(const double2 *x_full, int n_full, int64_t n_paths, double2 *x_out, uint8_t *slack_zero,
                             int has_next_slack, double slack_tol, cudaStream_t s)
{
    device_limits();
    if (n_paths <= 0) return cudaSuccess;
    int64_t grid = (n_paths + 255) / 256;
    if (grid > (int64_t)g_num_sms * 16) grid = (int64_t)g_num_sms * 16;
    drop_last_kernel<<<(unsigned)grid, 256, 0, s>>>(x_full, n_full, n_paths, x_out, slack_zero, has_next_slack,
                                                    slack_tol);
    return cudaGetLastError();
}

}  // namespace phc
