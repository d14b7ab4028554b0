// Allocation-free entry point: Morton keys and their stable sort into the
// caller's buffers, with all temporary memory taken from one fixed-size array
// that the library reserves when it is loaded.
//
// Who needs this: code that must not call cudaMalloc on its hot path, for
// example a real-time loop with a fixed device-memory budget (a cudaMalloc
// can block on the device and can fail part-way through a run), or a host
// application whose device allocator belongs to another framework (memory
// taken behind that allocator's back is memory it cannot hand out). Such a
// caller passes its own input and output buffers and gets the first stage of
// the octree build without the library allocating anything.
//
// The scratch is a file-scope __device__ array, so every GPU that loads the
// library holds it (NOALLOC_MAX_N * 12 bytes plus histograms, about 12.3 MB)
// until the process exits. Host code cannot use the array's name as a device
// address; its address is read with cudaGetSymbolAddress once per device, on
// the first call made with that device current.
#include <mutex>

#include "fmm_internal.cuh"

namespace fmm {

constexpr int64_t NOALLOC_MAX_N = 1 << 20;                       // largest n a call accepts
constexpr int64_t NOALLOC_TILES = NOALLOC_MAX_N / 4096;          // radix-sort tiles at that size
constexpr size_t NOALLOC_KEYS = sizeof(uint64_t) * NOALLOC_MAX_N; // ping-pong keys
constexpr size_t NOALLOC_PERM = sizeof(int) * NOALLOC_MAX_N;      // ping-pong indices
constexpr size_t NOALLOC_HIST = sizeof(unsigned) * 256 * NOALLOC_TILES;
constexpr size_t NOALLOC_BSUM = sizeof(unsigned) * 1024;
constexpr size_t NOALLOC_BYTES = NOALLOC_KEYS + NOALLOC_PERM + NOALLOC_HIST + NOALLOC_BSUM + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

namespace {
constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
unsigned char *g_ptr[MAX_DEVICES] = {};  // device address of the scratch, per device
int g_nsm[MAX_DEVICES] = {};
}  // namespace

}  // namespace fmm

extern "C" FMM_API int fmm_morton_sort_noalloc(const void *x, int64_t n, int dtype, uint64_t *keys, int32_t *perm,
                                               void *stream)
{
    using namespace fmm;
    if (!x || !keys || !perm) {
        set_error("fmm_morton_sort_noalloc: NULL pointer");
        return FMM_EINVAL;
    }
    if (dtype != FMM_F32 && dtype != FMM_F64) {
        set_error("fmm_morton_sort_noalloc: dtype must be FMM_F32 or FMM_F64 (device memory)");
        return FMM_EINVAL;
    }
    if (n < 1 || n > NOALLOC_MAX_N) {
        set_error("fmm_morton_sort_noalloc: n must be in [1, 1048576], the capacity of the static scratch");
        return FMM_EINVAL;
    }
    try {
        int dev = 0;
        FMM_CUDA_TRY(cudaGetDevice(&dev));
        if (dev < 0 || dev >= MAX_DEVICES) throw Error{FMM_ENODEV, "fmm_morton_sort_noalloc: device index out of range"};
        unsigned char *base;
        int nsm;
        {
            std::lock_guard<std::mutex> lk(g_mu);
            if (!g_ptr[dev]) {
                // once per device, with that device current
                void *p = nullptr;
                FMM_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
                int sm = 0;
                FMM_CUDA_TRY(cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev));
                g_ptr[dev] = static_cast<unsigned char *>(p);
                g_nsm[dev] = sm;
            }
            base = g_ptr[dev];
            nsm = g_nsm[dev];
        }
        uint64_t *ktmp = reinterpret_cast<uint64_t *>(base);
        int *ptmp = reinterpret_cast<int *>(base + NOALLOC_KEYS);
        unsigned *hist = reinterpret_cast<unsigned *>(base + NOALLOC_KEYS + NOALLOC_PERM);
        unsigned *bsum = reinterpret_cast<unsigned *>(base + NOALLOC_KEYS + NOALLOC_PERM + NOALLOC_HIST);
        Box *box = reinterpret_cast<Box *>(base + NOALLOC_KEYS + NOALLOC_PERM + NOALLOC_HIST + NOALLOC_BSUM);
        static_assert(sizeof(Box) <= 256, "root-cube scratch");
        morton_sort_into(x, n, dtype, keys, perm, ktmp, ptmp, hist, bsum, box, nsm, (cudaStream_t)stream);
        return FMM_OK;
    } catch (const Error &e) {
        set_error(e.msg);
        return e.code;
    }
}
