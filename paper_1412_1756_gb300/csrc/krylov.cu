// Inner GMRES of the characteristic-mode solver (Section IV: the inner
// solves with Z or X of the implicitly restarted Arnoldi method) on the
// device.  Vectors are complex FP32 in leaf order; a product is the plan's
// core pass on two real columns (real and imaginary part) combined into
// Z v or X v = Im(Z) v; the preconditioner is the same near-field strip
// kernel with the values of the sparse approximate inverse; inner products
// are accumulated in FP64; the (restart + 1) x restart Hessenberg matrix
// and its Givens rotations live on the host.
#include "krylov.h"
#include "device.h"
#include "plan_host.h"

#include <algorithm>
#include <cmath>
#include <vector>

namespace mlfma {
bool plan_product_view(mlfma_plan_t p, int prec, int64_t Bi, ProductArgs<float> *a32, ProductArgs<double> *a64, int *device,
                       int *max_batch, int64_t *n);
const PlanHost *plan_host(mlfma_plan_t p);

namespace {

constexpr int kDotBlocks = 120;
using cd = std::complex<double>;

#define KRYLOV_LOOP(i, n) \
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

inline int blocks_of(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8)); }

// xp [n][2] = (Re v, Im v)
__global__ void k_split(const float2 *v, float *xp, int64_t n)
{
    KRYLOV_LOOP(i, n)
    {
        const float2 a = v[i];
        xp[2 * i] = a.x;
        xp[2 * i + 1] = a.y;
    }
}

// yp [n][2] complex = (M Re v, M Im v) -> mode 0: M v; mode 1: Im(M Re v) + i Im(M Im v)
__global__ void k_combine(const float2 *yp, float2 *w, int64_t n, int mode)
{
    KRYLOV_LOOP(i, n)
    {
        const float2 a = yp[2 * i], c = yp[2 * i + 1];
        w[i] = mode == 0 ? make_float2(a.x - c.y, a.y + c.x) : make_float2(a.y, c.y);
    }
}

// part[j][block] = partial sums of conj(V_j) . w  (FP64)
__global__ void k_dots(const float2 *V, int64_t ld, const float2 *w, int64_t n, double2 *part)
{
    __shared__ double rs[256], is[256];
    const float2 *v = V + (int64_t)blockIdx.y * ld;
    double sr = 0, si = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 a = v[i], b = w[i];
        sr += (double)a.x * b.x + (double)a.y * b.y;
        si += (double)a.x * b.y - (double)a.y * b.x;
    }
    rs[threadIdx.x] = sr;
    is[threadIdx.x] = si;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) {
            rs[threadIdx.x] += rs[threadIdx.x + off];
            is[threadIdx.x] += is[threadIdx.x + off];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = make_double2(rs[0], is[0]);
}

__global__ void k_dots_reduce(const double2 *part, int nblk, double2 *h)
{
    __shared__ double rs[128], is[128];
    double sr = 0, si = 0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
        const double2 p = part[(int64_t)blockIdx.x * nblk + b];
        sr += p.x;
        si += p.y;
    }
    rs[threadIdx.x] = sr;
    is[threadIdx.x] = si;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) {
            rs[threadIdx.x] += rs[threadIdx.x + off];
            is[threadIdx.x] += is[threadIdx.x + off];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) h[blockIdx.x] = make_double2(rs[0], is[0]);
}

// out = sign * sum_j c_j V_j + (accumulate ? out : 0)
__global__ void k_lincomb(float2 *out, const float2 *V, int64_t ld, int nv, const double2 *c, int64_t n, float sign,
                          int accumulate)
{
    KRYLOV_LOOP(i, n)
    {
        float2 acc = accumulate ? out[i] : make_float2(0.f, 0.f);
        for (int j = 0; j < nv; ++j) {
            const float2 v = V[(int64_t)j * ld + i];
            const float cr = sign * (float)c[j].x, ci = sign * (float)c[j].y;
            acc.x += cr * v.x - ci * v.y;
            acc.y += cr * v.y + ci * v.x;
        }
        out[i] = acc;
    }
}

__global__ void k_scale(float2 *dst, const float2 *src, int64_t n, float s)
{
    KRYLOV_LOOP(i, n) dst[i] = make_float2(s * src[i].x, s * src[i].y);
}

__global__ void k_add(float2 *d, const float2 *z, int64_t n)
{
    KRYLOV_LOOP(i, n) d[i] = make_float2(d[i].x + z[i].x, d[i].y + z[i].y);
}

__global__ void k_sub(float2 *out, const float2 *a, const float2 *b, int64_t n)
{
    KRYLOV_LOOP(i, n) out[i] = make_float2(a[i].x - b[i].x, a[i].y - b[i].y);
}

void givens(cd x, cd y, double &c, cd &s)
{
    const double ax = std::abs(x), ay = std::abs(y);
    if (ay == 0) { c = 1; s = 0; return; }
    if (ax == 0) { c = 0; s = std::conj(y) / ay; return; }
    const double nr = std::hypot(ax, ay);
    c = ax / nr;
    s = (x / ax) * std::conj(y) / nr;
}

}  // namespace

class DeviceGmres {
  public:
    ProductArgs<float> aZ, aP;
    bool has_sai = false;
    int64_t n = 0;
    int restart = 0, device = 0;
    cudaStream_t s = nullptr;
    float2 *V = nullptr, *w = nullptr, *z = nullptr, *t = nullptr, *d = nullptr, *r = nullptr, *rr = nullptr;
    float2 *sai = nullptr;
    double2 *part = nullptr, *hd = nullptr;
    std::vector<int64_t> perm;
    std::vector<float2> stage;
    std::vector<double2> hh;

    ~DeviceGmres()
    {
        for (void *p : {(void *)V, (void *)w, (void *)z, (void *)t, (void *)d, (void *)r, (void *)rr, (void *)sai,
                        (void *)part, (void *)hd})
            if (p) cudaFree(p);
        if (s) cudaStreamDestroy(s);
    }

    cudaError_t product(const float2 *v, float2 *out, int mode)
    {
        cudaError_t e;
        k_split<<<blocks_of(n), 256, 0, s>>>(v, aZ.xp, n);
        CoreStreams cs{};
        cs.main = s;
        if ((e = launch_core<float>(aZ, cs, nullptr)) != cudaSuccess) return e;
        k_combine<<<blocks_of(n), 256, 0, s>>>(reinterpret_cast<const float2 *>(aZ.yp), out, n, mode);
        return cudaGetLastError();
    }

    cudaError_t precondition(const float2 *v, float2 *out)
    {
        if (!has_sai) return cudaMemcpyAsync(out, v, n * sizeof(float2), cudaMemcpyDeviceToDevice, s);
        cudaError_t e;
        k_split<<<blocks_of(n), 256, 0, s>>>(v, aP.xp, n);
        CoreStreams cs{};
        cs.main = s;
        if ((e = launch_core<float>(aP, cs, nullptr)) != cudaSuccess) return e;   // near-field stage only
        k_combine<<<blocks_of(n), 256, 0, s>>>(reinterpret_cast<const float2 *>(aP.yp), out, n, 0);
        return cudaGetLastError();
    }

    // h[0..nv) = V[0..nv)^H x, on the host
    cudaError_t dots(const float2 *Vb, int nv, const float2 *x)
    {
        k_dots<<<dim3(kDotBlocks, nv), 256, 0, s>>>(Vb, n, x, n, part);
        k_dots_reduce<<<nv, 128, 0, s>>>(part, kDotBlocks, hd);
        cudaError_t e = cudaMemcpyAsync(hh.data(), hd, nv * sizeof(double2), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return e;
        return cudaStreamSynchronize(s);
    }

    double norm(const float2 *x)
    {
        if (dots(x, 1, x) != cudaSuccess) return -1.0;
        return std::sqrt(std::max(0.0, hh[0].x));
    }
};

DeviceGmres *device_gmres_create(mlfma_plan_t p, const std::complex<double> *sai, int restart, std::string &err)
{
    ProductArgs<float> a32;
    int dev = 0, maxb = 0;
    int64_t n = 0;
    if (!plan_product_view(p, MLFMA_FP32, 0, &a32, nullptr, &dev, &maxb, &n)) {
        err = "device GMRES needs a device plan with FP32 set up";
        return nullptr;
    }
    if (maxb < 2) {
        err = "device GMRES needs max_batch >= 2";
        return nullptr;
    }
    const PlanHost *H = plan_host(p);
    DeviceGmres *g = new DeviceGmres();
    g->n = n;
    g->restart = restart;
    g->device = dev;
    g->perm = H->perm;
    g->stage.resize(n);
    g->hh.resize(restart + 2);
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
    cudaError_t e = cudaStreamCreateWithFlags(&g->s, cudaStreamNonBlocking);
    auto alloc = [&](void **ptr, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(ptr, bytes);
    };
    alloc((void **)&g->V, (size_t)(restart + 1) * n * sizeof(float2));
    for (float2 **q : {&g->w, &g->z, &g->t, &g->d, &g->r, &g->rr}) alloc((void **)q, (size_t)n * sizeof(float2));
    alloc((void **)&g->part, (size_t)(restart + 1) * kDotBlocks * sizeof(double2));
    alloc((void **)&g->hd, (size_t)(restart + 2) * sizeof(double2));
    g->aZ = a32;
    g->aZ.B = 2;
    g->aP = g->aZ;
    g->aP.coarsest = g->aP.leaf + 1;   // the near-field stage alone
    if (sai && e == cudaSuccess) {
        std::vector<float2> v((size_t)H->nnz);
        for (int64_t i = 0; i < H->nnz; ++i) v[i] = make_float2((float)sai[i].real(), (float)sai[i].imag());
        alloc((void **)&g->sai, v.size() * sizeof(float2));
        if (e == cudaSuccess) e = cudaMemcpy(g->sai, v.data(), v.size() * sizeof(float2), cudaMemcpyHostToDevice);
        g->aP.near_val = reinterpret_cast<const float *>(g->sai);
        g->has_sai = true;
    }
    if (prev != dev) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        err = std::string("device GMRES setup: ") + cudaGetErrorString(e);
        delete g;
        return nullptr;
    }
    return g;
}

void device_gmres_destroy(DeviceGmres *g) { delete g; }

int device_gmres_run(DeviceGmres *g, int mode, const std::complex<double> *rhost, std::complex<double> *dhost,
                     double target, int maxit, std::string &err)
{
    const int64_t n = g->n;
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != g->device) cudaSetDevice(g->device);
    auto done = [&](int ret) {
        if (prev != g->device) cudaSetDevice(prev);
        return ret;
    };
    cudaError_t e;
#define KTRY(x) do { if ((e = (x)) != cudaSuccess) { err = std::string("device GMRES: ") + cudaGetErrorString(e); return done(-1); } } while (0)
    for (int64_t i = 0; i < n; ++i) {
        const cd v = rhost[g->perm[i]];
        g->stage[i] = make_float2((float)v.real(), (float)v.imag());
    }
    KTRY(cudaMemcpyAsync(g->r, g->stage.data(), n * sizeof(float2), cudaMemcpyHostToDevice, g->s));
    KTRY(cudaMemcpyAsync(g->rr, g->r, n * sizeof(float2), cudaMemcpyDeviceToDevice, g->s));
    KTRY(cudaMemsetAsync(g->d, 0, n * sizeof(float2), g->s));
    double rn = g->norm(g->rr);
    if (rn < 0) {
        err = "device GMRES: norm failed";
        return done(-1);
    }
    int used = 0;
    const int m0 = g->restart;
    std::vector<cd> Hm((size_t)(m0 + 1) * m0), gv(m0 + 1), sn(m0), y;
    std::vector<double> cr(m0);
    while (used < maxit && rn > target) {
        const int m = std::min(m0, maxit - used);
        std::fill(Hm.begin(), Hm.end(), cd(0.0));
        std::fill(gv.begin(), gv.end(), cd(0.0));
        k_scale<<<blocks_of(n), 256, 0, g->s>>>(g->V, g->rr, n, (float)(1.0 / rn));
        gv[0] = rn;
        int k = 0;
        for (; k < m; ++k) {
            float2 *vk = g->V + (size_t)k * n, *vk1 = g->V + (size_t)(k + 1) * n;
            KTRY(g->precondition(vk, g->z));
            KTRY(g->product(g->z, vk1, mode));
            ++used;
            for (int pass = 0; pass < 2; ++pass) {   // classical Gram-Schmidt, twice
                KTRY(g->dots(g->V, k + 1, vk1));
                for (int j = 0; j <= k; ++j) Hm[(size_t)j * m + k] += cd(g->hh[j].x, g->hh[j].y);
                k_lincomb<<<blocks_of(n), 256, 0, g->s>>>(vk1, g->V, n, k + 1, g->hd, n, -1.f, 1);
            }
            const double hn = g->norm(vk1);
            if (hn < 0) {
                err = "device GMRES: norm failed";
                return done(-1);
            }
            Hm[(size_t)(k + 1) * m + k] = hn;
            if (hn > 0) k_scale<<<blocks_of(n), 256, 0, g->s>>>(vk1, vk1, n, (float)(1.0 / hn));
            for (int j = 0; j < k; ++j) {   // previous rotations
                const cd a = Hm[(size_t)j * m + k], bb = Hm[(size_t)(j + 1) * m + k];
                Hm[(size_t)j * m + k] = cr[j] * a + sn[j] * bb;
                Hm[(size_t)(j + 1) * m + k] = -std::conj(sn[j]) * a + cr[j] * bb;
            }
            double c;
            cd sr;
            givens(Hm[(size_t)k * m + k], Hm[(size_t)(k + 1) * m + k], c, sr);
            cr[k] = c;
            sn[k] = sr;
            Hm[(size_t)k * m + k] = c * Hm[(size_t)k * m + k] + sr * Hm[(size_t)(k + 1) * m + k];
            Hm[(size_t)(k + 1) * m + k] = 0.0;
            gv[k + 1] = -std::conj(sr) * gv[k];
            gv[k] = c * gv[k];
            if (std::abs(gv[k + 1]) <= target || used >= maxit) {
                ++k;
                break;
            }
        }
        // y = H^-1 g; d += P V y; true residual rr = r - M d
        y.assign(k, cd(0.0));
        for (int i = k - 1; i >= 0; --i) {
            cd sacc = gv[i];
            for (int j = i + 1; j < k; ++j) sacc -= Hm[(size_t)i * m + j] * y[j];
            y[i] = sacc / Hm[(size_t)i * m + i];
        }
        for (int j = 0; j < k; ++j) g->hh[j] = make_double2(y[j].real(), y[j].imag());
        KTRY(cudaMemcpyAsync(g->hd, g->hh.data(), k * sizeof(double2), cudaMemcpyHostToDevice, g->s));
        k_lincomb<<<blocks_of(n), 256, 0, g->s>>>(g->t, g->V, n, k, g->hd, n, 1.f, 0);
        KTRY(g->precondition(g->t, g->z));
        k_add<<<blocks_of(n), 256, 0, g->s>>>(g->d, g->z, n);
        KTRY(g->product(g->d, g->w, mode));
        k_sub<<<blocks_of(n), 256, 0, g->s>>>(g->rr, g->r, g->w, n);
        KTRY(cudaGetLastError());
        rn = g->norm(g->rr);
        if (rn < 0) {
            err = "device GMRES: norm failed";
            return done(-1);
        }
    }
    KTRY(cudaMemcpyAsync(g->stage.data(), g->d, n * sizeof(float2), cudaMemcpyDeviceToHost, g->s));
    KTRY(cudaStreamSynchronize(g->s));
    for (int64_t i = 0; i < n; ++i) dhost[g->perm[i]] = cd(g->stage[i].x, g->stage[i].y);
#undef KTRY
    return done(used);
}

}  // namespace mlfma
