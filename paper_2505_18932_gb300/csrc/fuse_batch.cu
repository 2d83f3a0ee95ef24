// Batched fusion: many (frame, target) items in one persistent launch.
#include "fuse_march.cuh"

namespace gvs {
namespace {

// Many (frame, target) items in one persistent launch: each warp takes the
// next bundle index from a global counter until every item's bundles are
// taken, and marches it with that item's arguments.  No warp ever waits on
// another; the counter is reset before each launch.
template <int KMAX, typename MT, typename T>
__global__ void __launch_bounds__(32 * FZ_WARPS, GVS_FUSE_MIN_BLOCKS)
    fuse_batch_kernel(const BatchItem *__restrict__ items, int n_items, int total, unsigned *__restrict__ counter) {
    // each warp keeps its current item's arguments in shared memory (read there by the
    // march, instead of from global memory at every use)
    __shared__ FuseArgs s_args[FZ_WARPS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    static_assert(sizeof(FuseArgs) % sizeof(int) == 0, "copied as words");
    // the warp's current item and its bundle range: a warp's bundles come in increasing
    // order, mostly from the same item, so the table is searched only on a change of item
    int cur = -1, cur_begin = 0, cur_end = 0;
    for (;;) {
        int b = 0;
        if (lane == 0) b = (int)atomicAdd(counter, 1u);
        b = __shfl_sync(0xffffffffu, b, 0);
        if (b >= total) break;
        if (b < cur_begin || b >= cur_end) {
            int lo = 0, hi = n_items - 1;  // last item whose first bundle is <= b
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (items[mid].bundle_begin <= b) lo = mid; else hi = mid - 1;
            }
            cur = lo;
            cur_begin = items[lo].bundle_begin;
            cur_end = lo + 1 < n_items ? items[lo + 1].bundle_begin : total;
            // every lane has left the previous march (the shuffle above synchronised them)
            const int *src = reinterpret_cast<const int *>(&items[cur].args);
            int *dst = reinterpret_cast<int *>(&s_args[warp]);
            for (int i = lane; i < (int)(sizeof(FuseArgs) / sizeof(int)); i += 32) dst[i] = __ldg(&src[i]);
            __syncwarp();
        }
        march_bundle<KMAX, MT, T, false, false>(s_args[warp], b - cur_begin, lane);
    }
}

template <int KMAX, typename MT, typename T>
void launch_batch_t(const BatchItem *items, int n_items, int total, unsigned *counter, cudaStream_t st) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fuse_batch_kernel<KMAX, MT, T>, 32 * FZ_WARPS, 0) !=
            cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const int64_t want = ((int64_t)total + FZ_WARPS - 1) / FZ_WARPS;
    int64_t grid = (int64_t)per_sm * device_sm_count();
    if (grid > want) grid = want;
    if (grid < 1) grid = 1;
    fuse_batch_kernel<KMAX, MT, T><<<(unsigned)grid, 32 * FZ_WARPS, 0, st>>>(items, n_items, total, counter);
}

template <int KMAX, typename MT, typename T>
struct BatchLaunch {
    static void run(const BatchItem *items, int n, int total, unsigned *counter, cudaStream_t st) {
        launch_batch_t<KMAX, MT, T>(items, n, total, counter, st);
    }
};

}  // namespace

cudaError_t launch_fuse_batch(const BatchItem *items, int n_items, int total, unsigned *counter, int K, int map_dtype,
                              int variant, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    by_kmax<BatchLaunch>(K, map_dtype, variant, items, n_items, total, counter, st);
    return cudaGetLastError();
}
GVS_BOUNDS_TAKE_FN(bounds_take_fuse_batch)

}  // namespace gvs
