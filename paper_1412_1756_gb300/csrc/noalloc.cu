// mlfma_matvec_noalloc: the product y = Z x with every per-call scratch
// buffer (leaf-order columns and the outgoing/incoming fields of every
// level) carved from one file-scope static device array instead of the
// plan's own buffers.  The call allocates nothing and captures no graph: it
// launches the same kernels in order on the caller's stream.
#include "../../include/mlfma.h"
#include "device.h"

#include <mutex>
#include <string>

namespace mlfma {
bool plan_product_view(mlfma_plan_t p, int prec, int64_t Bi, ProductArgs<float> *a32, ProductArgs<double> *a64,
                       int *device, int *max_batch, int64_t *n);
void set_last_error(const std::string &msg);
}  // namespace mlfma

using namespace mlfma;

namespace {

// The static scratch.  Every GPU that loads this library holds it until the
// process exits.  In host code `g_noalloc_scratch` is only a host-side
// stand-in for the symbol, never a device address: kernels get the address
// that cudaGetSymbolAddress returns for the current device.
constexpr size_t kScratchBytes = (size_t)MLFMA_NOALLOC_SCRATCH_BYTES;
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
void *g_addr[kMaxDevices] = {};

// Device address of the static scratch on `dev` (which must be current),
// looked up once per device and kept for the life of the process: after a
// cudaDeviceReset of that device (a new primary context) the kept address is
// stale, so the entry point must not be called across a reset.
cudaError_t scratch_address(int dev, void **out)
{
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (!g_addr[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = ptr;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

mlfma_status fail(mlfma_status st, const std::string &msg)
{
    set_last_error(msg);
    return st;
}

// Lays the per-call buffers of a product with B real columns out in the
// scratch starting at `base` (nullptr: only count); returns the bytes used.
template <class R>
size_t carve(ProductArgs<R> &a, int B, unsigned char *base)
{
    size_t off = 0;
    auto take = [&](size_t bytes) -> R * {
        R *p = base ? reinterpret_cast<R *>(base + off) : nullptr;
        off = align256(off + bytes);
        return p;
    };
    a.xp = take((size_t)a.n * B * sizeof(R));
    a.yp = take((size_t)a.n * B * 2 * sizeof(R));
    for (int l = 2; l <= a.leaf; ++l) {
        const size_t f = (size_t)a.lv[l].nbox * 2 * a.lv[l].K * B * 2 * sizeof(R);
        a.lv[l].S = take(f);
        a.lv[l].G = take(f);
    }
    return off;
}

template <class R>
mlfma_status run(ProductArgs<R> a, const void *x, int xc, void *y, int64_t B, int64_t Bi, void *scratch,
                 cudaStream_t s)
{
    const size_t need = carve<R>(a, (int)Bi, nullptr);
    if (need > kScratchBytes)
        return fail(MLFMA_EINVAL, "mlfma_matvec_noalloc: this product needs " + std::to_string(need) +
                                      " bytes of scratch; the static scratch holds " + std::to_string(kScratchBytes) +
                                      " bytes (use fewer columns or mlfma_matvec)");
    a.B = (int)Bi;
    carve<R>(a, (int)Bi, static_cast<unsigned char *>(scratch));
    CoreStreams serial{};
    serial.main = s;   // no side streams: every stage in order on the caller's stream
    cudaError_t e;
    if ((e = launch_prepare<R>(a, x, xc, (int)B, 0, s)) != cudaSuccess ||
        (e = launch_core<R>(a, serial, nullptr)) != cudaSuccess ||
        (e = launch_finalize<R>(a, y, xc, (int)B, 0, s)) != cudaSuccess)
        return fail(MLFMA_ECUDA, std::string("mlfma_matvec_noalloc: ") + cudaGetErrorString(e));
    return MLFMA_OK;
}

}  // namespace

extern "C" mlfma_status mlfma_matvec_noalloc(mlfma_plan_t plan, const void *x, int x_is_complex, void *y, int64_t B,
                                             int prec, void *stream)
{
    if (!plan) return fail(MLFMA_EINVAL, "plan is NULL");
    if (!x || !y) return fail(MLFMA_EINVAL, "x or y is NULL");
    if (B < 1) return fail(MLFMA_EINVAL, "B must be >= 1");
    if (prec != MLFMA_FP32 && prec != MLFMA_FP64) return fail(MLFMA_EINVAL, "unknown precision");
    ProductArgs<float> a32;
    ProductArgs<double> a64;
    int dev = -1, max_batch = 0;
    int64_t n = 0;
    const int64_t Bi = B * (x_is_complex ? 2 : 1);
    if (mlfma_num_unknowns(plan, &n) != MLFMA_OK) return MLFMA_EINVAL;
    const int64_t rsz = prec == MLFMA_FP64 ? 8 : 4;
    if (byte_ranges_overlap(x, n * Bi * rsz, y, n * B * 2 * rsz))
        return fail(MLFMA_EINVAL, "x and y must not overlap");
    if (!plan_product_view(plan, prec, Bi, &a32, &a64, &dev, &max_batch, &n))
        return fail(MLFMA_EINVAL, "plan is host-only or lacks this precision");
    if (Bi > max_batch) return fail(MLFMA_EINVAL, "B exceeds the plan's max_batch");
    if (dev < 0 || dev >= kMaxDevices) return fail(MLFMA_EINVAL, "device ordinal out of range");
    int prev = -1;
    cudaError_t e = cudaGetDevice(&prev);
    if (e != cudaSuccess) return fail(MLFMA_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (prev != dev && (e = cudaSetDevice(dev)) != cudaSuccess)
        return fail(MLFMA_ECUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    void *scratch = nullptr;
    mlfma_status st;
    if ((e = scratch_address(dev, &scratch)) != cudaSuccess) {
        st = fail(MLFMA_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    } else if (prec == MLFMA_FP32) {
        st = run<float>(a32, x, x_is_complex, y, B, Bi, scratch, static_cast<cudaStream_t>(stream));
    } else {
        st = run<double>(a64, x, x_is_complex, y, B, Bi, scratch, static_cast<cudaStream_t>(stream));
    }
    if (prev != dev) cudaSetDevice(prev);
    return st;
}
