// track_multi.cu -- launcher of the multi-system tracker (systems of
// different structure, one per warp at a time); a translation unit of its
// own so it compiles in parallel with the other modes.
#include "track_impl.cuh"

namespace phc {

// Threads per block: shared memory per thread plus a table region per warp.
static int multi_block_threads(const TrackLaunch &L, int n, int block_threads)
{
    const size_t per =
        thread_smem_bytes(n, true, L.o.precision == PHC_PREC_FP32_INTERIOR) + (size_t)L.warp_table_bytes / 32;
    long fit = (long)g_smem_optin / (long)per;
    int bt = (int)((fit / 32) * 32);
    if (bt > 256) bt = 256;
    if (block_threads > 0 && block_threads < bt) bt = block_threads;
    return bt < 32 ? 0 : bt;
}

cudaError_t launch_multi(const TrackLaunch &L, int n, int block_threads, int max_blocks, cudaStream_t s)
{
    device_limits();
    if (L.n_multi <= 0) return cudaSuccess;
    const int bt = multi_block_threads(L, n, block_threads);
    if (bt == 0) return cudaErrorInvalidConfiguration;
#define PHC_CALL_MULTI(NN) launch_track_n<NN, MODE_MULTI>(L, bt, max_blocks, L.n_paths, s)
    PHC_DISPATCH_N(n, PHC_CALL_MULTI)
#undef PHC_CALL_MULTI
}

int64_t multi_lanes(const TrackLaunch &L, int n, int block_threads, int max_blocks)
{
    device_limits();
    const int bt = multi_block_threads(L, n, block_threads);
    if (bt == 0) return -1;
    switch (n) {
    case 1: return lanes_n<1, MODE_MULTI>(L, bt, max_blocks);
    case 2: return lanes_n<2, MODE_MULTI>(L, bt, max_blocks);
    case 3: return lanes_n<3, MODE_MULTI>(L, bt, max_blocks);
    case 4: return lanes_n<4, MODE_MULTI>(L, bt, max_blocks);
    case 5: return lanes_n<5, MODE_MULTI>(L, bt, max_blocks);
    case 6: return lanes_n<6, MODE_MULTI>(L, bt, max_blocks);
    case 7: return lanes_n<7, MODE_MULTI>(L, bt, max_blocks);
    case 8: return lanes_n<8, MODE_MULTI>(L, bt, max_blocks);
    case 9: return lanes_n<9, MODE_MULTI>(L, bt, max_blocks);
    case 10: return lanes_n<10, MODE_MULTI>(L, bt, max_blocks);
    case 11: return lanes_n<11, MODE_MULTI>(L, bt, max_blocks);
    case 12: return lanes_n<12, MODE_MULTI>(L, bt, max_blocks);
    default: return -1;
    }
}

}  // namespace phc
