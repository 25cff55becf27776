// noalloc.cu -- rubix_spaxel_sort_noalloc: spaxel assignment + stable sort by
// spaxel whose scratch memory lives in a fixed, file-scope device array, so the
// call itself never allocates device memory.
//
// Who needs this: callers that may not allocate device memory on their own,
// because another allocator owns the device's memory budget (a framework's
// caching allocator or a memory pool sized at start-up, where a stray
// cudaMalloc can fail or fragment the pool), or because the call sits in a
// latency-critical loop where cudaMalloc/cudaFree would add an implicit device
// synchronisation. They pass their own input and output buffers; the
// intermediate arrays of the sort live in `g_noalloc_scratch` below.
//
// Limits: at most kNoallocMaxParticles particles and at most
// kNoallocMaxKeys - 1 spaxels (nx * ny); larger problems are rejected with
// RUBIX_ERR_INVALID_ARG. The array (about 4.3 MB) is held on every device that
// loads the library until the process exits.
//
// Sharing: every call, on every stream, uses the same array and leaves its
// contents behind. Every scratch word the kernels read is first written by the
// same call, so nothing needs clearing between calls; but two calls whose work
// overlaps on the GPU (different streams, or different host threads, without
// ordering between them) race on the array and give wrong results.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/rubix.h"
#include "common.cuh"
#include "kernels.h"
#include "engine.h"

namespace rubix {

constexpr long long kNoallocMaxParticles = 1ll << 18;   // 262144
constexpr int kNoallocMaxKeys = 1 << 18;                // keys in [0, nx*ny]
constexpr long long kNoallocTiles = (kNoallocMaxParticles + 4095) / 4096;
// keys, keys_tmp, vals_tmp, sorted keys, then the sort's digit counts/offsets/scan scratch
constexpr long long kNoallocSortInts = 2 * kNoallocTiles * 512 + (kNoallocTiles * 512 + 4095) / 4096 + 1 + 16;
constexpr long long kNoallocInts = 4 * kNoallocMaxParticles + kNoallocSortInts;

static __device__ __align__(256) int g_noalloc_scratch[kNoallocInts];

}  // namespace rubix

using namespace rubix;

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
int* g_noalloc_ptr[kMaxDevices] = {};
}  // namespace

namespace rubix {
void set_last_error(const char* msg);  // the thread-local message behind rubix_last_error_message()
}

static long long n_or_1(long long n) { return n > 0 ? n : 1; }

// The host-side name `g_noalloc_scratch` is only a stand-in for the device
// array: its device address is fetched once per device (with that device
// current) and handed to the kernels.
static rubix_status noalloc_scratch(int dev, int** out) {
    if (dev < 0 || dev >= kMaxDevices) return RUBIX_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            char m[160];
            snprintf(m, sizeof(m), "cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            set_last_error(m);
            return RUBIX_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = static_cast<int*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return RUBIX_OK;
}

extern "C" rubix_status rubix_spaxel_sort_noalloc(const rubix_particles* p, const rubix_telescope* tel,
                                                  int32_t* perm_out, int32_t* seg_off_out, void* stream) {
    auto bad = [](const char* m) {
        set_last_error(m);
        return (rubix_status)RUBIX_ERR_INVALID_ARG;
    };
    if (!p || !tel || !perm_out || !seg_off_out) return bad("NULL argument");
    if (!p->on_device) return bad("particles must be device pointers (on_device = 1)");
    if (p->n < 0) return bad("n < 0");
    if (p->n > kNoallocMaxParticles) return bad("n exceeds the no-allocation limit of 262144 particles");
    if (tel->nx < 1 || tel->ny < 1 || (long long)tel->nx * tel->ny + 1 > kNoallocMaxKeys)
        return bad("nx*ny exceeds the no-allocation limit of 262143 spaxels");
    if (!(tel->spaxel_size > 0.0)) return bad("spaxel_size must be > 0");
    if (p->n > 0 && (!p->x || !p->y)) return bad("x, y required");
    if (p->n > 0 && !p->preprojected && !p->z) return bad("z required when not preprojected");

    // the sort's scratch layout (tiles, digit buckets, scan tiles) must fit
    // the fixed array; a change of those constants shows up here, not as an
    // overrun
    if ((long long)sort_scratch_ints(n_or_1(p->n)) > kNoallocSortInts) {
        set_last_error("internal: the sort needs more scratch than the no-allocation array holds");
        return RUBIX_ERR_UNSUPPORTED;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        set_last_error("no CUDA device");
        return RUBIX_ERR_CUDA;
    }
    int* base = nullptr;
    rubix_status s = noalloc_scratch(dev, &base);
    if (s != RUBIX_OK) return s;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const long long n = p->n;
    const int n_keys = tel->nx * tel->ny + 1;
    int* keys = base;
    int* keys_tmp = base + kNoallocMaxParticles;
    int* vals_tmp = base + 2 * kNoallocMaxParticles;
    int* skeys = base + 3 * kNoallocMaxParticles;
    int* sort_scratch = base + 4 * kNoallocMaxParticles;

    AssignParams A{};
    A.n = n;
    A.x = p->x;
    A.y = p->y;
    A.z = p->z;
    A.vy = nullptr;
    A.vz = nullptr;
    A.v_los = nullptr;
    A.preprojected = p->preprojected ? 1 : 0;
    orientation_matrix(p->inclination, p->azimuth, p->position_angle, A.R, A.Di, A.Da);
    A.x_lo = (-0.5 * (double)tel->nx) * tel->spaxel_size;
    A.y_lo = (-0.5 * (double)tel->ny) * tel->spaxel_size;
    A.inv_size = 1.0 / tel->spaxel_size;
    A.nx = tel->nx;
    A.ny = tel->ny;
    A.key = keys;
    A.pin_out = nullptr;
    launch_assign(A, st);
    launch_sort_by_key(keys, n, n_keys, keys_tmp, vals_tmp, skeys, perm_out, seg_off_out, sort_scratch, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        char m[160];
        snprintf(m, sizeof(m), "launch failed: %s", cudaGetErrorString(e));
        set_last_error(m);
        return RUBIX_ERR_CUDA;
    }
    return RUBIX_OK;
}
