// noalloc.cu -- scg_tv_static: the TV norm for callers that cannot allocate
// device memory.
//
// scg_tv needs a small device workspace (solver state, problem descriptor, a
// counter and one block of FP64 partial sums per image tile) that the caller
// allocates.  Some callers cannot do that: a plug-in living inside a host
// application whose memory pool owns the whole device, a real-time loop whose
// rules forbid allocator calls because they may block or fail, or a program
// with a fixed device-memory budget decided at start-up.  This entry point keeps
// that scratch in a fixed array that the library itself defines in device
// memory, so the caller passes only the image and the output location.
//
// The array is a file-scope __device__ variable of kStaticBytes (about 1 MiB):
// it exists on every GPU that loads the library, from the load until the
// process exits, and serves images up to kStaticMaxN x kStaticMaxN.  Every
// call uses the same array, which keeps the last call's contents; the parts
// that must start at zero (state, counter) are cleared by each call, on the
// caller's stream.  Two calls that may run at the same time on the GPU (for
// example from two streams) race on the array and give undefined results.
//
// Host code cannot use the array's name as a device address: on the host it
// names a stand-in object, and a kernel given that address would fault or, on
// systems where the GPU can reach host memory, silently use the wrong memory.
// The device address is therefore fetched with cudaGetSymbolAddress, once per
// device, with that device current, on the first call made on the device.  The
// address belongs to the device's current context: scg_release() forgets it,
// so after a context is destroyed (cudaDeviceReset) the caller calls
// scg_release() and the next call looks the address up again.
#include <string.h>

#include <mutex>

#include "scg_kernels.h"

using namespace scg;

namespace {

constexpr int kStaticMaxN = 1024;   // largest image side this entry point accepts
constexpr int kStaticTiles = ((kStaticMaxN + kTileH - 1) / kTileH) * ((kStaticMaxN + kTileW - 1) / kTileW);
constexpr size_t al256(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t kOffState = 0;
constexpr size_t kOffProb = al256(sizeof(DevState));
constexpr size_t kOffCounter = kOffProb + al256(sizeof(Prob<double>));
constexpr size_t kOffPartials = kOffCounter + 256;
constexpr size_t kStaticBytes = kOffPartials + sizeof(double) * kSlots * (size_t)kStaticTiles;

static __device__ __align__(256) unsigned char g_tv_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_scratch_dev[kMaxDevices];   // device address of g_tv_scratch, per device

// Device address of the scratch array on the current device (set up on the
// first call on that device).
int scratch_address(unsigned char** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SCG_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return SCG_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_tv_scratch) != cudaSuccess || !p) return SCG_ERR_CUDA;
        g_scratch_dev[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_dev[dev];
    return SCG_OK;
}

}  // namespace

namespace scg {
// Forget the cached scratch addresses (called by scg_release).
void noalloc_forget() {
    std::lock_guard<std::mutex> lk(g_mu);
    for (int d = 0; d < kMaxDevices; ++d) g_scratch_dev[d] = nullptr;
}
}  // namespace scg

namespace {

template <typename T>
int tv_static_impl(int n, const void* x, double* tv_out, cudaStream_t s) {
    unsigned char* base = nullptr;
    int rc = scratch_address(&base);
    if (rc != SCG_OK) return rc;
    Prob<T> P;
    memset(&P, 0, sizeof(P));
    P.n = n;
    P.na = 1;
    P.nb = 1;
    P.tiles_x = (n + kTileW - 1) / kTileW;
    P.cnt_img = ((n + kTileH - 1) / kTileH) * P.tiles_x;
    P.img[IB_AUX] = const_cast<T*>(static_cast<const T*>(x));
    P.partials = reinterpret_cast<double*>(base + kOffPartials);
    P.part_cap = kStaticTiles;
    P.counter = reinterpret_cast<unsigned*>(base + kOffCounter);
    P.st = reinterpret_cast<DevState*>(base + kOffState);
    P.trace = tv_out;
    P.trace_rows = 1;
    if (cudaMemsetAsync(base + kOffState, 0, sizeof(DevState), s) != cudaSuccess) return SCG_ERR_CUDA;
    if (cudaMemsetAsync(base + kOffCounter, 0, 256, s) != cudaSuccess) return SCG_ERR_CUDA;
    if (cudaMemcpyAsync(base + kOffProb, &P, sizeof(P), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return SCG_ERR_CUDA;
    launch_tvgrad<T>(reinterpret_cast<const Prob<T>*>(base + kOffProb), nullptr, P.cnt_img, IB_AUX, 0, 0,
                     FIN_TV, s);
    if (cudaGetLastError() != cudaSuccess) return SCG_ERR_CUDA;
    return SCG_OK;
}

}  // namespace

extern "C" int scg_tv_static(int n, int precision, const void* x, double* tv_out, void* stream) {
    if (n < 2 || !x || !tv_out) return SCG_ERR_INVALID;
    if (n > kStaticMaxN) return SCG_ERR_UNSUPPORTED;
    if (precision != SCG_F32 && precision != SCG_F64) return SCG_ERR_UNSUPPORTED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    return precision == SCG_F64 ? tv_static_impl<double>(n, x, tv_out, s)
                                : tv_static_impl<float>(n, x, tv_out, s);
}
