// Outer Arnoldi basis of the characteristic-mode solver on the device
// (Section IV: the implicitly restarted Arnoldi method on Eq. (SEP1) or
// (SEP)).  The m + 1 basis vectors are complex FP64 in device memory; the
// classical Gram-Schmidt orthogonalisation (two passes), the normalisation,
// the implicit restart's recombination of the basis and the Ritz vectors run
// as FP64 kernels.  Inner products are reduced per CTA on the device and the
// partial sums added in FP64 on the host, in a fixed order.  The small
// ncv x ncv Hessenberg matrix and its eigenproblem stay on the host.
#include "krylov.h"
#include "device.h"

#include <algorithm>
#include <vector>

namespace mlfma {
bool plan_product_view(mlfma_plan_t p, int prec, int64_t Bi, ProductArgs<float> *a32, ProductArgs<double> *a64, int *device,
                       int *max_batch, int64_t *n);

namespace {

constexpr int kBlocks = 96;   // CTAs per inner product
using cd = std::complex<double>;

#define ARN_LOOP(i, n) \
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// part[j][block] = this CTA's share of conj(V_j) . w, for the rows j < gridDim.y
__global__ void k_arn_dots(const double2 *V, int64_t n, const double2 *w, double2 *part)
{
    __shared__ double rs[256], is[256];
    const double2 *v = V + (int64_t)blockIdx.y * n;
    double sr = 0, si = 0;
    ARN_LOOP(i, n)
    {
        const double2 a = v[i], b = w[i];
        sr = fma(a.x, b.x, fma(a.y, b.y, sr));
        si = fma(a.x, b.y, fma(-a.y, b.x, si));
    }
    rs[threadIdx.x] = sr;
    is[threadIdx.x] = si;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            rs[threadIdx.x] += rs[threadIdx.x + s];
            is[threadIdx.x] += is[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = make_double2(rs[0], is[0]);
}

// w -= sum_{j < rows} h_j V_j
__global__ void k_arn_subtract(const double2 *V, int64_t n, int rows, const double2 *h, double2 *w)
{
    ARN_LOOP(i, n)
    {
        double2 a = w[i];
        for (int j = 0; j < rows; ++j) {
            const double2 c = h[j], v = V[(int64_t)j * n + i];
            a.x -= c.x * v.x - c.y * v.y;
            a.y -= c.x * v.y + c.y * v.x;
        }
        w[i] = a;
    }
}

__global__ void k_arn_scale(const double2 *w, double s, double2 *out, int64_t n)
{
    ARN_LOOP(i, n) out[i] = make_double2(w[i].x * s, w[i].y * s);
}

// out[c] = sum_{j < rows} coef[j][c] V_j for c < cols
__global__ void k_arn_combine(const double2 *V, int64_t n, int rows, int cols, const double2 *coef, double2 *out)
{
    ARN_LOOP(i, n)
    {
        for (int c = 0; c < cols; ++c) {
            double2 a = make_double2(0.0, 0.0);
            for (int j = 0; j < rows; ++j) {
                const double2 q = coef[(int64_t)j * cols + c], v = V[(int64_t)j * n + i];
                a.x += q.x * v.x - q.y * v.y;
                a.y += q.x * v.y + q.y * v.x;
            }
            out[(int64_t)c * n + i] = a;
        }
    }
}

inline int grid_of(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8)); }

}  // namespace

class DeviceArnoldi {
  public:
    int64_t n = 0;
    int m = 0, device = 0;
    double2 *V = nullptr;      // [m + 1][n] basis
    double2 *S = nullptr;      // [m + 1][n] recombination scratch
    double2 *w = nullptr;      // [n]
    double2 *part = nullptr;   // [m + 1][kBlocks]
    double2 *coef = nullptr;   // [(m + 1) * (m + 1)]
    std::vector<double2> hpart;

    bool ok(cudaError_t e, const char *what, std::string &err)
    {
        if (e == cudaSuccess) return true;
        err = std::string("device Arnoldi: ") + what + ": " + cudaGetErrorString(e);
        return false;
    }
    // h[j] = conj(V_j) . w for j < rows, summed on the host in block order
    bool dots(const double2 *vec, int rows, cd *h, std::string &err)
    {
        dim3 grid(kBlocks, rows);
        k_arn_dots<<<grid, 256>>>(V, n, vec, part);
        if (!ok(cudaGetLastError(), "dots", err)) return false;
        hpart.resize((size_t)rows * kBlocks);
        if (!ok(cudaMemcpy(hpart.data(), part, hpart.size() * sizeof(double2), cudaMemcpyDeviceToHost), "dots", err))
            return false;
        for (int j = 0; j < rows; ++j) {
            double r = 0, i = 0;
            for (int b = 0; b < kBlocks; ++b) {
                r += hpart[(size_t)j * kBlocks + b].x;
                i += hpart[(size_t)j * kBlocks + b].y;
            }
            h[j] = cd(r, i);
        }
        return true;
    }
    // ||vec|| via a dot product of vec with itself (rows of the basis are not touched)
    bool norm(const double2 *vec, double &out, std::string &err)
    {
        k_arn_dots<<<dim3(kBlocks, 1), 256>>>(vec, n, vec, part);
        if (!ok(cudaGetLastError(), "norm", err)) return false;
        hpart.resize(kBlocks);
        if (!ok(cudaMemcpy(hpart.data(), part, kBlocks * sizeof(double2), cudaMemcpyDeviceToHost), "norm", err))
            return false;
        double r = 0;
        for (int b = 0; b < kBlocks; ++b) r += hpart[b].x;
        out = std::sqrt(std::max(r, 0.0));
        return true;
    }
};

DeviceArnoldi *arnoldi_create(mlfma_plan_t p, int64_t n, int m, std::string &err)
{
    int device = 0, maxb = 0;
    int64_t np = 0;
    if (!plan_product_view(p, MLFMA_FP64, 1, nullptr, nullptr, &device, &maxb, &np) &&
        !plan_product_view(p, MLFMA_FP32, 1, nullptr, nullptr, &device, &maxb, &np)) {
        err = "device Arnoldi: the plan has no device products";
        return nullptr;
    }
    if (cudaSetDevice(device) != cudaSuccess) {
        err = "device Arnoldi: cannot select the plan's device";
        return nullptr;
    }
    auto *a = new DeviceArnoldi;
    a->n = n;
    a->m = m;
    a->device = device;
    const size_t vb = (size_t)(m + 1) * n * sizeof(double2);
    if (!a->ok(cudaMalloc(&a->V, vb), "alloc", err) || !a->ok(cudaMalloc(&a->S, vb), "alloc", err) ||
        !a->ok(cudaMalloc(&a->w, (size_t)n * sizeof(double2)), "alloc", err) ||
        !a->ok(cudaMalloc(&a->part, (size_t)(m + 1) * kBlocks * sizeof(double2)), "alloc", err) ||
        !a->ok(cudaMalloc(&a->coef, (size_t)(m + 1) * (m + 1) * sizeof(double2)), "alloc", err)) {
        arnoldi_destroy(a);
        return nullptr;
    }
    return a;
}

void arnoldi_destroy(DeviceArnoldi *a)
{
    if (!a) return;
    cudaSetDevice(a->device);
    cudaFree(a->V);
    cudaFree(a->S);
    cudaFree(a->w);
    cudaFree(a->part);
    cudaFree(a->coef);
    delete a;
}

bool arnoldi_set(DeviceArnoldi *a, int j, const cd *v, std::string &err)
{
    return a->ok(cudaMemcpy(a->V + (int64_t)j * a->n, v, (size_t)a->n * sizeof(double2), cudaMemcpyHostToDevice),
                 "set", err);
}

bool arnoldi_get(DeviceArnoldi *a, int j, cd *v, std::string &err)
{
    return a->ok(cudaMemcpy(v, a->V + (int64_t)j * a->n, (size_t)a->n * sizeof(double2), cudaMemcpyDeviceToHost),
                 "get", err);
}

bool arnoldi_extend(DeviceArnoldi *a, int j, const cd *wh, cd *h, double *hn, cd *out, std::string &err)
{
    const int64_t n = a->n;
    if (!a->ok(cudaMemcpy(a->w, wh, (size_t)n * sizeof(double2), cudaMemcpyHostToDevice), "extend", err)) return false;
    std::vector<cd> c(j + 1);
    for (int pass = 0; pass < 2; ++pass) {   // classical Gram-Schmidt, twice
        if (!a->dots(a->w, j + 1, c.data(), err)) return false;
        for (int i = 0; i <= j; ++i) h[i] += c[i];
        if (!a->ok(cudaMemcpy(a->coef, c.data(), (size_t)(j + 1) * sizeof(double2), cudaMemcpyHostToDevice), "extend",
                   err))
            return false;
        k_arn_subtract<<<grid_of(n), 256>>>(a->V, n, j + 1, a->coef, a->w);
        if (!a->ok(cudaGetLastError(), "extend", err)) return false;
    }
    if (!a->norm(a->w, *hn, err)) return false;
    k_arn_scale<<<grid_of(n), 256>>>(a->w, *hn > 0 ? 1.0 / *hn : 0.0, a->V + (int64_t)(j + 1) * n, n);
    if (!a->ok(cudaGetLastError(), "extend", err)) return false;
    return out ? arnoldi_get(a, j + 1, out, err) : true;
}

bool arnoldi_recombine(DeviceArnoldi *a, int rows, int cols, const cd *coef, std::string &err)
{
    const int64_t n = a->n;
    if (!a->ok(cudaMemcpy(a->coef, coef, (size_t)rows * cols * sizeof(double2), cudaMemcpyHostToDevice), "restart", err))
        return false;
    k_arn_combine<<<grid_of(n), 256>>>(a->V, n, rows, cols, a->coef, a->S);
    if (!a->ok(cudaGetLastError(), "restart", err)) return false;
    return a->ok(cudaMemcpy(a->V, a->S, (size_t)cols * n * sizeof(double2), cudaMemcpyDeviceToDevice), "restart", err);
}

bool arnoldi_normalise(DeviceArnoldi *a, int j, double *nrm, std::string &err)
{
    double2 *v = a->V + (int64_t)j * a->n;
    if (!a->norm(v, *nrm, err)) return false;
    k_arn_scale<<<grid_of(a->n), 256>>>(v, *nrm > 0 ? 1.0 / *nrm : 0.0, v, a->n);
    return a->ok(cudaGetLastError(), "normalise", err);
}

bool arnoldi_combine(DeviceArnoldi *a, int rows, int cols, const cd *coef, cd *out, std::string &err)
{
    const int64_t n = a->n;
    if (!a->ok(cudaMemcpy(a->coef, coef, (size_t)rows * cols * sizeof(double2), cudaMemcpyHostToDevice), "Ritz", err))
        return false;
    k_arn_combine<<<grid_of(n), 256>>>(a->V, n, rows, cols, a->coef, a->S);
    if (!a->ok(cudaGetLastError(), "Ritz", err)) return false;
    return a->ok(cudaMemcpy(out, a->S, (size_t)cols * n * sizeof(double2), cudaMemcpyDeviceToHost), "Ritz", err);
}

}  // namespace mlfma
