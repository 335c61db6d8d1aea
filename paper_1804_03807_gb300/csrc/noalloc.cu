// noalloc.cu -- phc_track_paths_noalloc: path tracking without any device
// allocation during the call.
//
// phc_track_paths may call cudaMalloc: for the per-path records when the
// caller passes no statistics array, and for the hand-off records of the tail
// kernel (both grow with the launch and are kept in the handle).  Some callers
// cannot allocate while they run: a process whose device memory is owned by
// another allocator (a framework's caching allocator that reserved the free
// HBM up front, so cudaMalloc fails or fragments its pool), or a
// latency-critical serving loop that allocates everything at start-up and
// must not stall in the allocator afterwards.  This entry point takes its
// scratch -- the path-queue counter, the hand-off counters, the hand-off
// records and, when stats_out is NULL, the per-path records the
// classification pass reads -- from one file-scope device array of fixed size
// instead.
//
// Properties a caller must know:
//  * The array is static device memory: every GPU that loads the library
//    holds NOALLOC_SCRATCH_BYTES of it until the process exits.
//  * Set-up: the first call on a device (with that device current) looks up
//    the array's device address with cudaGetSymbolAddress; that first call
//    should come before any stream capture.
//  * Every call shares the one array and it keeps the last call's contents;
//    the counters are cleared at the start of each call.  Calls that overlap
//    on the GPU (other streams, other threads) race on it: serialise them.
//  * With stats_out == NULL, n_paths may not exceed PHC_NOALLOC_MAX_PATHS.
//  * The tail hand-off (opts.tail_drain) keeps at most
//    PHC_NOALLOC_MAX_HANDOFF paths: it starts once no more than that many
//    of the tracker's threads still hold a path (later than tail_drain alone
//    would start it on launches of more threads), and the tracker runs
//    without the compaction of running paths (opts.compact is ignored).
//    Results are the same either way; only the time changes.
#include <mutex>

#include "phc_internal.h"

namespace phc {
// implemented in phc_api.cpp: the device view of a handle's total-degree
// homotopy and start tables, its hand-off counters, and option checking
int handle_track_view(phc_homotopy *h, const phc_opts &o, TrackLaunch *L);
unsigned long long *handle_tail_counters(phc_homotopy *h);
int handle_num_paths(const phc_homotopy *h, int64_t *out);
int check_options(const phc_opts &o);
int set_error(int code, const char *msg);
}  // namespace phc

// Layout of the scratch: the path-queue counter at byte 0, the four hand-off
// counters (records written, idle threads, tail queue, tail units) at byte 64,
// the hand-off records from byte 256, then the per-path records.
#define NOALLOC_HEAD_BYTES 256
#define NOALLOC_HANDOFF_BYTES ((size_t)PHC_NOALLOC_MAX_HANDOFF * sizeof(phc::Handoff))
#define NOALLOC_STATS_OFFSET (NOALLOC_HEAD_BYTES + ((NOALLOC_HANDOFF_BYTES + 255) & ~(size_t)255))
#define NOALLOC_SCRATCH_BYTES (NOALLOC_STATS_OFFSET + (size_t)PHC_NOALLOC_MAX_PATHS * sizeof(phc_path_stats))

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

static std::mutex g_setup_mutex;
static void *g_scratch_ptr[64];  // device address per device ordinal

// Device address of g_noalloc_scratch on the current device (set-up once per
// device).  The host-side name of the array is not a device address.
static int scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return phc::set_error(PHC_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= 64) return phc::set_error(PHC_EUNSUPPORTED, "device ordinal above 63");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return phc::set_error(PHC_ECUDA, "cudaGetSymbolAddress of the no-allocation scratch failed");
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return PHC_OK;
}

extern "C" int phc_track_paths_noalloc(phc_homotopy *h, int64_t first, int64_t n, const phc_opts *opts,
                                       phc_cd *x_out, int8_t *cls_out, phc_path_stats *stats_out, void *stream)
{
    if (!h) return phc::set_error(PHC_EINVAL, "NULL handle");
    int64_t total = 0;
    int rc = phc::handle_num_paths(h, &total);
    if (rc) return rc;
    if (n < 0 || first < 0 || first + n > total)
        return phc::set_error(PHC_EINVAL, "path range outside [0, number of paths)");
    if (n == 0) return PHC_OK;
    if (!x_out || !cls_out) return phc::set_error(PHC_EINVAL, "NULL output array");
    if (!stats_out && n > PHC_NOALLOC_MAX_PATHS)
        return phc::set_error(PHC_EUNSUPPORTED,
                              "phc_track_paths_noalloc: n_paths above PHC_NOALLOC_MAX_PATHS with stats_out == NULL "
                              "(pass a stats array or split the range)");
    phc_opts o;
    if (opts) o = *opts; else phc_default_opts(&o);
    rc = phc::check_options(o);
    if (rc) return rc;
    void *base = nullptr;
    rc = scratch_address(&base);
    if (rc) return rc;
    unsigned char *b = static_cast<unsigned char *>(base);
    unsigned long long *counter = reinterpret_cast<unsigned long long *>(b);
    unsigned long long *tailc = reinterpret_cast<unsigned long long *>(b + 64);
    phc_path_stats *st = stats_out ? stats_out : reinterpret_cast<phc_path_stats *>(b + NOALLOC_STATS_OFFSET);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(b, 0, NOALLOC_HEAD_BYTES, s);
    if (e != cudaSuccess) return phc::set_error(PHC_ECUDA, cudaGetErrorString(e));
    // the handle's own hand-off counters describe its last phc_track_paths
    // call; this call is not one, so phc_tail_paths reports 0 after it
    if (unsigned long long *hc = phc::handle_tail_counters(h)) {
        e = cudaMemsetAsync(hc, 0, 4 * sizeof(unsigned long long), s);
        if (e != cudaSuccess) return phc::set_error(PHC_ECUDA, cudaGetErrorString(e));
    }

    phc::TrackLaunch L{};
    rc = phc::handle_track_view(h, o, &L);
    if (rc) return rc;
    L.start_mode = 0;
    L.starts = nullptr;
    L.first = first;
    L.n_paths = n;
    L.x_out = reinterpret_cast<double2 *>(x_out);
    L.stats = st;
    L.qhead = counter;
    L.o = o;
    // no compaction here: the hand-off cap relies on idle lanes staying idle
    // (running paths <= lanes - idle_n at every moment), which moving paths
    // between lanes only keeps up to a transient
    L.compact = 0;
    const bool tail = o.tail_drain > 0.0 && phc::tail_supported(L.tab);
    if (tail) {
        L.handoff = reinterpret_cast<phc::Handoff *>(b + NOALLOC_HEAD_BYTES);
        L.handoff_n = tailc;
        L.idle_n = tailc + 1;
        L.tail_q = tailc + 2;
        L.tail_units = tailc + 3;
        L.drain_frac = o.tail_drain;
        L.handoff_cap = PHC_NOALLOC_MAX_HANDOFF;
    }
    e = phc::launch_track(L, o.block_threads, o.max_blocks, s);
    if (e != cudaSuccess) return phc::set_error(PHC_ECUDA, cudaGetErrorString(e));
    if (tail) {
        e = phc::launch_tail(L, o.max_blocks, s);
        if (e != cudaSuccess) return phc::set_error(PHC_ECUDA, cudaGetErrorString(e));
    }
    phc::ClassifyLaunch C{};
    C.tab = L.tab;
    C.tab.f32 = 0;
    C.n_paths = n;
    C.x = L.x_out;
    C.stats = st;
    C.cls = cls_out;
    C.o = o;
    e = phc::launch_classify(C, s);
    if (e != cudaSuccess) return phc::set_error(PHC_ECUDA, cudaGetErrorString(e));
    return PHC_OK;
}
