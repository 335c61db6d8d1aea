// track_pipe.cu -- launcher of the pipelined tracker (top stage and cascade
// stage in one launch); a translation unit of its own so it compiles in
// parallel with the other modes.
#include "track_impl.cuh"

namespace phc {

cudaError_t launch_pipeline(const TrackLaunch &L, int block_threads, int max_blocks, cudaStream_t s)
{
    device_limits();
    if (L.n_paths <= 0) return cudaSuccess;
    const size_t tb = table_smem_bytes(L.tab) + table_smem_bytes(L.tab2);
    const int bt = track_block_threads(L.tab.n, tb, block_threads, true, L.o.precision == PHC_PREC_FP32_INTERIOR,
                                       localp_pipe_of(L.tab.n));
    if (bt == 0) return cudaErrorInvalidConfiguration;
#define PHC_CALL_PIPE(NN) launch_track_n<NN, MODE_PIPE>(L, bt, max_blocks, L.n_paths, s)
    PHC_DISPATCH_N(L.tab.n, PHC_CALL_PIPE)
#undef PHC_CALL_PIPE
}

int64_t pipe_lanes(const TrackLaunch &L, int block_threads, int max_blocks)
{
    device_limits();
    const size_t tb = table_smem_bytes(L.tab) + table_smem_bytes(L.tab2);
    const int bt = track_block_threads(L.tab.n, tb, block_threads, true, L.o.precision == PHC_PREC_FP32_INTERIOR,
                                       localp_pipe_of(L.tab.n));
    if (bt == 0) return -1;
    switch (L.tab.n) {
    case 1: return lanes_n<1, MODE_PIPE>(L, bt, max_blocks);
    case 2: return lanes_n<2, MODE_PIPE>(L, bt, max_blocks);
    case 3: return lanes_n<3, MODE_PIPE>(L, bt, max_blocks);
    case 4: return lanes_n<4, MODE_PIPE>(L, bt, max_blocks);
    case 5: return lanes_n<5, MODE_PIPE>(L, bt, max_blocks);
    case 6: return lanes_n<6, MODE_PIPE>(L, bt, max_blocks);
    case 7: return lanes_n<7, MODE_PIPE>(L, bt, max_blocks);
    case 8: return lanes_n<8, MODE_PIPE>(L, bt, max_blocks);
    case 9: return lanes_n<9, MODE_PIPE>(L, bt, max_blocks);
    case 10: return lanes_n<10, MODE_PIPE>(L, bt, max_blocks);
    case 11: return lanes_n<11, MODE_PIPE>(L, bt, max_blocks);
    case 12: return lanes_n<12, MODE_PIPE>(L, bt, max_blocks);
    default: return -1;
    }
}

}  // namespace phc
