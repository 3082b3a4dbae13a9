// hmat_matvec_noalloc: the H-matrix product of an uploaded handle with every
// scratch buffer taken from one static device array, so that the call itself
// allocates no memory.
//
// Who needs it: callers that must not allocate device memory at the time they
// run the product -- real-time or latency-critical loops that cannot pay for a
// cudaMalloc (it can synchronise the device and take milliseconds), and host
// programs or plugins whose device memory is owned by another allocator or
// memory budget (a framework's caching allocator, a fixed reservation) that
// they may not go around.  They create the handle once at set-up (hmat_upload
// allocates then) and afterwards call only this entry point.
//
// The scratch is the source-vector operand copy, the projection partial sums
// and the phase-2 operand buffers; the handle's own copies of those buffers are
// not used, so this entry point never races with the handle's other calls on
// the same stream -- but every call on every handle shares the one static array.
#include <cuda_runtime.h>

#include <mutex>

#include "handle.h"

using namespace hmat_internal;

namespace {

constexpr size_t kNoallocScratchBytes = HMAT_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// Every GPU that loads the library holds this array until the process exits.
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_addr_mutex;
void *g_addr[kMaxDevices] = {};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Device address of the array on the current device; looked up once per device
// (cudaGetSymbolAddress with that device current), then cached.
int scratch_address(int dev, void **out) {
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (!g_addr[dev]) {
        void *p = nullptr;
        CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return HMAT_OK;
}

// Device (or managed) memory the kernels on `device` may use: device memory of
// another GPU is refused, the kernels would read or write a peer's memory.
bool on_device(const void *p, int device) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeDevice) return a.device == device;
    return a.type == cudaMemoryTypeManaged;
}

size_t scratch_bytes_for(const hmat_t *h) {
    const HmatSegment &g = h->seg[0];
    const size_t ob = operand_bytes(g.store), pb = partial_bytes(g.store);
    return align256((size_t)h->n * ob) + align256((size_t)(g.partials_n > 0 ? g.partials_n : 1) * pb) +
           align256((size_t)(g.glen > 0 ? g.glen : 1) * ob);
}

}  // namespace

extern "C" int hmat_matvec_noalloc(hmat_handle h, const double *x, double *y, void *stream) {
    if (!h || !x || !y || x == y) return HMAT_ERR_ARG;
    if (int e = take_status(h)) return e;  // a bounded wait of an earlier product ran out
    int dev = -1;
    CK(cudaGetDevice(&dev));
    if (dev != h->device || dev < 0 || dev >= kMaxDevices) return HMAT_ERR_ARG;
    if (!on_device(x, dev) || !on_device(y, dev)) return HMAT_ERR_ARG;  // no staging buffers: this device's memory only
    if (h->nseg != 1) return HMAT_ERR_UNSUPPORTED;            // the paper's two-segment variants
    const size_t need = scratch_bytes_for(h);
    if (need > kNoallocScratchBytes) return HMAT_ERR_UNSUPPORTED;
    void *base = nullptr;
    int st = scratch_address(dev, &base);
    if (st != HMAT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const HmatSegment &g = h->seg[0];
    const size_t ob = operand_bytes(g.store);
    DevPanels P = g.P;
    char *b = (char *)base;
    P.xs = b;
    P.part = b + align256((size_t)h->n * ob);
    P.g = b + align256((size_t)h->n * ob) + align256((size_t)(g.partials_n > 0 ? g.partials_n : 1) *
                                                      partial_bytes(g.store));
    // the array keeps the previous call's contents: the padding slots of the
    // operand buffers must read zero, every other slot is rewritten below
    CK(cudaMemsetAsync(P.g, 0, (size_t)(g.glen > 0 ? g.glen : 1) * ob, s));
    launch_prep(g.store, g.ix, x, h->perm, P.xs, s);
    launch_phase1(g.store, g.ix, P, nullptr, 0, s);
    launch_reduce(g.store, g.ix, P, nullptr, 0, s);
    launch_phase2(g.store, g.ix, P, y, h->perm, 0, nullptr, 0, s);
    CK(cudaGetLastError());
    return HMAT_OK;
}
