// Block inner solves of the characteristic-mode solver on the device: the p
// real right-hand sides of X D = B (X = Im Z) advance together, one MLFMA
// product of p real columns per step, each column with its own Krylov basis,
// Hessenberg matrix and Givens rotations (restarted GMRES, right-
// preconditioned by the real sparse approximate inverse of the near part of
// X, Section IV).  Vectors are FP32 in leaf order, [n][p] with the column
// index innermost (the product's input layout); inner products are
// accumulated in FP64; the small Hessenberg problems live on the host.
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

constexpr int kRowBlocks = 96;   // row blocks of the column-dot kernel

#define BLOCK_LOOP(i, n) \
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

inline int grid_of(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8)); }

// part[(j p + c) nrb + blk] = sum over the CTA's rows i of V_j[i][c] w[i][c].
// A warp reads 32 adjacent columns of one row; 8 warps per CTA take
// interleaved rows; grid (nrb, nv, ceil(p / 32)).  Each thread accumulates
// in FP32 with compensation: a product a b is split exactly into its rounded
// value pr and error fma(a, b, -pr), the running sum takes pr by TwoSum
// (Knuth: the rounding error of s + pr is recovered exactly) and a second
// FP32 accumulator collects both errors, so the thread's sum carries about
// twice the FP32 precision at FP32 ALU cost; the two accumulators are
// widened to FP64 only for the reduction across threads.
__global__ void __launch_bounds__(256) k_col_dots(const float *V, int64_t ld, const float *w, int64_t n, int p,
                                                  double *part)
{
    __shared__ double red[8][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int c = blockIdx.z * 32 + tx;
    const float *v = V + (int64_t)blockIdx.y * ld;
    float s = 0.f, err = 0.f;
    if (c < p)
        for (int64_t i = (int64_t)blockIdx.x * 8 + ty; i < n; i += (int64_t)gridDim.x * 8) {
            const float a = v[i * p + c], b = w[i * p + c];
            const float pr = a * b;
            const float pe = fmaf(a, b, -pr);
            const float t = s + pr;
            const float z = t - s;
            err += ((s - (t - z)) + (pr - z)) + pe;
            s = t;
        }
    red[ty][tx] = (double)s + (double)err;
    __syncthreads();
    if (ty == 0 && c < p) {
        double t = 0;
        for (int r = 0; r < 8; ++r) t += red[r][tx];
        part[((int64_t)blockIdx.y * p + c) * gridDim.x + blockIdx.x] = t;
    }
}

// h[t] = sum_b part[t nrb + b],  t = j p + c
__global__ void k_col_dots_reduce(const double *part, int nrb, int64_t m, double *h)
{
    BLOCK_LOOP(t, m)
    {
        double s = 0;
        for (int b = 0; b < nrb; ++b) s += part[t * nrb + b];
        h[t] = s;
    }
}

// out[i][c] = (acc ? out[i][c] : 0) + sign * sum_{j < nv} coef[j p + c] V_j[i][c],
// with the coefficients narrowed to FP32 once (k_narrow) rather than per
// element.
__global__ void k_col_lincomb(float *out, const float *V, int64_t ld, int nv, const float *coef, int64_t n, int p,
                              float sign, int acc)
{
    BLOCK_LOOP(e, n * p)
    {
        const int c = (int)(e % p);
        float s = 0.f;
        for (int j = 0; j < nv; ++j) s = fmaf(coef[(int64_t)j * p + c], V[(int64_t)j * ld + e], s);
        out[e] = (acc ? out[e] : 0.f) + sign * s;
    }
}

__global__ void k_narrow(float *dst, const double *src, int64_t n)
{
    BLOCK_LOOP(e, n) dst[e] = (float)src[e];
}

// dst[i][c] = f[c] src[i][c]
__global__ void k_col_scale(float *dst, const float *src, const double *f, int64_t n, int p)
{
    BLOCK_LOOP(e, n * p) dst[e] = (float)f[e % p] * src[e];
}

// dst = real (im = 0) or imaginary (im = 1) part of the complex product output
__global__ void k_take_part(float *dst, const float2 *yp, int64_t total, int im)
{
    BLOCK_LOOP(e, total) dst[e] = im ? yp[e].y : yp[e].x;
}

__global__ void k_accumulate(float *d, const float *z, int64_t total)
{
    BLOCK_LOOP(e, total) d[e] += z[e];
}

__global__ void k_difference(float *out, const float *a, const float *b, int64_t total)
{
    BLOCK_LOOP(e, total) out[e] = a[e] - b[e];
}

// Real Givens rotation [c s; -s c] with [c s; -s c] [x; y] = [r; 0].
void rotation(double x, double y, double &c, double &s)
{
    if (y == 0) { c = 1; s = 0; return; }
    const double r = std::hypot(x, y);
    c = x / r;
    s = y / r;
}

}  // namespace

class BlockGmres {
  public:
    ProductArgs<float> aZ, aP;
    bool has_sai = false;
    int64_t n = 0;
    int p = 0, restart = 0, device = 0;
    cudaStream_t s = nullptr;
    float *V = nullptr;   // restart + 1 blocks of [n][p]
    float *w = nullptr, *t = nullptr, *d = nullptr, *r = nullptr, *rr = nullptr;
    float2 *sai = nullptr;
    double *part = nullptr, *hd = nullptr, *cf = nullptr;
    float *cf32 = nullptr;   // coefficients narrowed for k_col_lincomb
    std::vector<int64_t> perm;
    std::vector<float> stage;
    std::vector<double> hh;

    ~BlockGmres()
    {
        for (void *q : {(void *)V, (void *)w, (void *)t, (void *)d, (void *)r, (void *)rr, (void *)sai, (void *)part,
                        (void *)hd, (void *)cf, (void *)cf32})
            if (q) cudaFree(q);
        if (s) cudaStreamDestroy(s);
    }

    int64_t size() const { return n * p; }

    // out = X v: the full product of the p real columns, imaginary part
    cudaError_t apply_x(const float *v, float *out)
    {
        cudaError_t e = cudaMemcpyAsync(aZ.xp, v, size() * sizeof(float), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
        CoreStreams cs{};
        cs.main = s;
        if ((e = launch_core<float>(aZ, cs, nullptr)) != cudaSuccess) return e;
        k_take_part<<<grid_of(size()), 256, 0, s>>>(out, reinterpret_cast<const float2 *>(aZ.yp), size(), 1);
        return cudaGetLastError();
    }

    // out = P v: the near-field stage alone with the (real) SAI values
    cudaError_t precondition(const float *v, float *out)
    {
        if (!has_sai) return cudaMemcpyAsync(out, v, size() * sizeof(float), cudaMemcpyDeviceToDevice, s);
        cudaError_t e = cudaMemcpyAsync(aP.xp, v, size() * sizeof(float), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
        CoreStreams cs{};
        cs.main = s;
        if ((e = launch_core<float>(aP, cs, nullptr)) != cudaSuccess) return e;
        k_take_part<<<grid_of(size()), 256, 0, s>>>(out, reinterpret_cast<const float2 *>(aP.yp), size(), 0);
        return cudaGetLastError();
    }

    // hh[j p + c] = V_j[:, c] . x[:, c] for j < nv (host, after a stream
    // sync); the same values stay on the device in hd
    cudaError_t dots(const float *Vb, int nv, const float *x)
    {
        k_col_dots<<<dim3(kRowBlocks, nv, (p + 31) / 32), 256, 0, s>>>(Vb, size(), x, n, p, part);
        k_col_dots_reduce<<<grid_of((int64_t)nv * p), 256, 0, s>>>(part, kRowBlocks, (int64_t)nv * p, hd);
        cudaError_t e = cudaMemcpyAsync(hh.data(), hd, (size_t)nv * p * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return e;
        return cudaStreamSynchronize(s);
    }

    cudaError_t norms(const float *x, std::vector<double> &out)
    {
        cudaError_t e = dots(x, 1, x);
        if (e != cudaSuccess) return e;
        for (int c = 0; c < p; ++c) out[c] = std::sqrt(std::max(0.0, hh[c]));
        return cudaSuccess;
    }

    // upload host coefficients (count doubles) to cf
    cudaError_t upload(const std::vector<double> &h, size_t count)
    {
        return cudaMemcpyAsync(cf, h.data(), count * sizeof(double), cudaMemcpyHostToDevice, s);
    }
};

BlockGmres *block_gmres_create(mlfma_plan_t p, const std::complex<double> *sai, int restart, int cols,
                               std::string &err)
{
    ProductArgs<float> a32;
    int dev = 0, maxb = 0;
    int64_t n = 0;
    if (!plan_product_view(p, MLFMA_FP32, 0, &a32, nullptr, &dev, &maxb, &n)) {
        err = "block GMRES needs a device plan with FP32 set up";
        return nullptr;
    }
    if (cols < 1 || cols > maxb) {
        err = "block GMRES: the block size must be in 1..max_batch";
        return nullptr;
    }
    if (restart < 1) {
        err = "block GMRES: restart must be >= 1";
        return nullptr;
    }
    const PlanHost *H = plan_host(p);
    BlockGmres *g = new BlockGmres();
    g->n = n;
    g->p = cols;
    g->restart = restart;
    g->device = dev;
    g->perm = H->perm;
    g->stage.resize((size_t)n * cols);
    g->hh.resize((size_t)(restart + 1) * cols);
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
    cudaError_t e = cudaStreamCreateWithFlags(&g->s, cudaStreamNonBlocking);
    auto alloc = [&](void **ptr, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(ptr, bytes);
    };
    const size_t blk = (size_t)n * cols * sizeof(float);
    alloc((void **)&g->V, (size_t)(restart + 1) * blk);
    for (float **q : {&g->w, &g->t, &g->d, &g->r, &g->rr}) alloc((void **)q, blk);
    alloc((void **)&g->part, (size_t)(restart + 1) * cols * kRowBlocks * sizeof(double));
    alloc((void **)&g->hd, (size_t)(restart + 1) * cols * sizeof(double));
    alloc((void **)&g->cf, (size_t)(restart + 1) * cols * sizeof(double));
    alloc((void **)&g->cf32, (size_t)(restart + 1) * cols * sizeof(float));
    g->aZ = a32;
    g->aZ.B = cols;
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
        err = std::string("block GMRES setup: ") + cudaGetErrorString(e);
        delete g;
        return nullptr;
    }
    return g;
}

void block_gmres_destroy(BlockGmres *g) { delete g; }

int block_gmres_run(BlockGmres *g, const double *bh, double *dh, int guess, double tol, int maxit, int *conv,
                    double *relres, std::string &err)
{
    const int64_t n = g->n, np = g->size();
    const int p = g->p, m0 = g->restart;
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != g->device) cudaSetDevice(g->device);
    auto done = [&](int ret) {
        if (prev != g->device) cudaSetDevice(prev);
        return ret;
    };
    cudaError_t e;
#define BTRY(x) do { if ((e = (x)) != cudaSuccess) { err = std::string("block GMRES: ") + cudaGetErrorString(e); return done(-1); } } while (0)
    for (int64_t i = 0; i < n; ++i) {
        const double *src = bh + g->perm[i] * p;
        for (int c = 0; c < p; ++c) g->stage[(size_t)i * p + c] = (float)src[c];
    }
    BTRY(cudaMemcpyAsync(g->r, g->stage.data(), np * sizeof(float), cudaMemcpyHostToDevice, g->s));
    std::vector<double> rn(p), bn(p), target(p), hn(p), f((size_t)(m0 + 1) * p), y;
    BTRY(g->norms(g->r, bn));
    if (guess) {   // d = the caller's D, rr = b - X d
        BTRY(cudaStreamSynchronize(g->s));   // the staging buffer is reused
        for (int64_t i = 0; i < n; ++i) {
            const double *src = dh + g->perm[i] * p;
            for (int c = 0; c < p; ++c) g->stage[(size_t)i * p + c] = (float)src[c];
        }
        BTRY(cudaMemcpyAsync(g->d, g->stage.data(), np * sizeof(float), cudaMemcpyHostToDevice, g->s));
        BTRY(g->apply_x(g->d, g->w));
        k_difference<<<grid_of(np), 256, 0, g->s>>>(g->rr, g->r, g->w, np);
        BTRY(cudaGetLastError());
    } else {
        BTRY(cudaMemcpyAsync(g->rr, g->r, np * sizeof(float), cudaMemcpyDeviceToDevice, g->s));
        BTRY(cudaMemsetAsync(g->d, 0, np * sizeof(float), g->s));
    }
    BTRY(g->norms(g->rr, rn));
    for (int c = 0; c < p; ++c) target[c] = tol * bn[c];
    std::vector<char> fin(p), active(p);
    for (int c = 0; c < p; ++c) fin[c] = rn[c] <= target[c];
    // per column: Hessenberg matrix ((m0 + 1) x m0, row-major), right-hand
    // side of the small least-squares problem, rotations, steps taken
    std::vector<double> Hm((size_t)p * (m0 + 1) * m0), gv((size_t)p * (m0 + 1)), cr((size_t)p * m0),
        sr((size_t)p * m0);
    std::vector<int> kc(p);
    auto h = [&](int c, int i, int j) -> double & { return Hm[((size_t)c * (m0 + 1) + i) * m0 + j]; };
    auto all_fin = [&]() {
        for (int c = 0; c < p; ++c)
            if (!fin[c]) return false;
        return true;
    };
    int used = 0;
    while (used < maxit && !all_fin()) {
        const int m = std::min(m0, maxit - used);
        std::fill(Hm.begin(), Hm.end(), 0.0);
        std::fill(gv.begin(), gv.end(), 0.0);
        for (int c = 0; c < p; ++c) {
            active[c] = !fin[c];
            kc[c] = 0;
            f[c] = active[c] ? 1.0 / rn[c] : 0.0;   // finished columns carry zero vectors
            gv[(size_t)c * (m0 + 1)] = active[c] ? rn[c] : 0.0;
        }
        BTRY(g->upload(f, p));
        k_col_scale<<<grid_of(np), 256, 0, g->s>>>(g->V, g->rr, g->cf, n, p);
        int steps = 0;
        for (int k = 0; k < m; ++k) {
            float *vk = g->V + (size_t)k * np, *vk1 = g->V + (size_t)(k + 1) * np;
            BTRY(g->precondition(vk, g->t));
            BTRY(g->apply_x(g->t, vk1));
            ++used;
            for (int pass = 0; pass < 2; ++pass) {   // classical Gram-Schmidt, twice, column by column
                BTRY(g->dots(g->V, k + 1, vk1));
                for (int c = 0; c < p; ++c)
                    if (active[c])
                        for (int j = 0; j <= k; ++j) h(c, j, k) += g->hh[(size_t)j * p + c];
                k_narrow<<<grid_of((int64_t)(k + 1) * p), 256, 0, g->s>>>(g->cf32, g->hd, (int64_t)(k + 1) * p);
                k_col_lincomb<<<grid_of(np), 256, 0, g->s>>>(vk1, g->V, np, k + 1, g->cf32, n, p, -1.f, 1);
            }
            BTRY(g->norms(vk1, hn));
            for (int c = 0; c < p; ++c) f[c] = active[c] && hn[c] > 0 ? 1.0 / hn[c] : 0.0;
            BTRY(g->upload(f, p));
            k_col_scale<<<grid_of(np), 256, 0, g->s>>>(vk1, vk1, g->cf, n, p);
            steps = k + 1;
            bool any = false;
            for (int c = 0; c < p; ++c) {
                if (!active[c]) continue;
                h(c, k + 1, k) = hn[c];
                double *cc = &cr[(size_t)c * m0], *ss = &sr[(size_t)c * m0], *gg = &gv[(size_t)c * (m0 + 1)];
                for (int j = 0; j < k; ++j) {   // previous rotations
                    const double a = h(c, j, k), b = h(c, j + 1, k);
                    h(c, j, k) = cc[j] * a + ss[j] * b;
                    h(c, j + 1, k) = -ss[j] * a + cc[j] * b;
                }
                rotation(h(c, k, k), h(c, k + 1, k), cc[k], ss[k]);
                h(c, k, k) = cc[k] * h(c, k, k) + ss[k] * h(c, k + 1, k);
                h(c, k + 1, k) = 0.0;
                gg[k + 1] = -ss[k] * gg[k];
                gg[k] = cc[k] * gg[k];
                kc[c] = k + 1;
                if (std::abs(gg[k + 1]) <= target[c] || hn[c] == 0) active[c] = 0;
                else any = true;
            }
            if (!any || used >= maxit) break;
        }
        // y_c = H_c^-1 g_c over the column's own steps; d += P (V y)
        std::fill(f.begin(), f.begin() + (size_t)steps * p, 0.0);
        for (int c = 0; c < p; ++c) {
            const int kk = kc[c];
            const double *gg = &gv[(size_t)c * (m0 + 1)];
            y.assign(kk, 0.0);
            for (int i = kk - 1; i >= 0; --i) {
                double acc = gg[i];
                for (int j = i + 1; j < kk; ++j) acc -= h(c, i, j) * y[j];
                y[i] = h(c, i, i) != 0 ? acc / h(c, i, i) : 0.0;
            }
            for (int j = 0; j < kk; ++j) f[(size_t)j * p + c] = y[j];
        }
        if (steps > 0) {
            BTRY(g->upload(f, (size_t)steps * p));
            k_narrow<<<grid_of((int64_t)steps * p), 256, 0, g->s>>>(g->cf32, g->cf, (int64_t)steps * p);
            k_col_lincomb<<<grid_of(np), 256, 0, g->s>>>(g->t, g->V, np, steps, g->cf32, n, p, 1.f, 0);
            BTRY(g->precondition(g->t, g->w));
            k_accumulate<<<grid_of(np), 256, 0, g->s>>>(g->d, g->w, np);
        }
        // true residual of every column
        BTRY(g->apply_x(g->d, g->w));
        k_difference<<<grid_of(np), 256, 0, g->s>>>(g->rr, g->r, g->w, np);
        BTRY(cudaGetLastError());
        BTRY(g->norms(g->rr, rn));
        for (int c = 0; c < p; ++c) fin[c] = rn[c] <= target[c];
    }
    BTRY(cudaMemcpyAsync(g->stage.data(), g->d, np * sizeof(float), cudaMemcpyDeviceToHost, g->s));
    BTRY(cudaStreamSynchronize(g->s));
    for (int64_t i = 0; i < n; ++i) {
        double *dst = dh + g->perm[i] * p;
        for (int c = 0; c < p; ++c) dst[c] = g->stage[(size_t)i * p + c];
    }
    for (int c = 0; c < p; ++c) {
        conv[c] = fin[c] ? 1 : 0;
        if (relres) relres[c] = bn[c] > 0 ? rn[c] / bn[c] : 0.0;
    }
#undef BTRY
    return done(used);
}

}  // namespace mlfma
