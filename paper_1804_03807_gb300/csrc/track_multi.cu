// track_multi.cu -- launcher of the multi-system tracker (systems of
// different structure, one per warp at a time); a translation unit of its
// own so it compiles in parallel with the other modes.
#include "track_impl.cuh"

namespace phc {

cudaError_t launch_multi(const TrackLaunch &L, int n, int block_threads, int max_blocks, cudaStream_t s)
{
    device_limits();
    if (L.n_multi <= 0) return cudaSuccess;
    // shared memory per thread plus a table region per warp
    const size_t per =
        thread_smem_bytes(n, true, L.o.precision == PHC_PREC_FP32_INTERIOR) + (size_t)L.warp_table_bytes / 32;
    long fit = (long)g_smem_optin / (long)per;
    int bt = (int)((fit / 32) * 32);
    if (bt > 256) bt = 256;
    if (block_threads > 0 && block_threads < bt) bt = block_threads;
    if (bt < 32) return cudaErrorInvalidConfiguration;
#define PHC_CALL_MULTI(NN) launch_track_n<NN, MODE_MULTI>(L, bt, max_blocks, L.n_paths, s)
    PHC_DISPATCH_N(n, PHC_CALL_MULTI)
#undef PHC_CALL_MULTI
}

}  // namespace phc
