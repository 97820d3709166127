// Reception of FP32 fields at the leaf level (the disaggregation of Section
// III: y_i += sum_q w_q conj(V_i(q)) . G_m(q) over the samples q of leaf box
// m, both tangential components, for the unknowns i of the box; w_q carries
// the quadrature weight and the far constant).
//
// One CTA per (leaf box, chunk of 2 NCP columns), 256 threads: thread =
// (column pair, row group), rows i = group + k * groups.  Tiles of QT
// samples: the field tile is loaded into registers one tile ahead, scaled by
// w_q and stored to shared memory (so w costs nothing in the inner loop); the
// pattern tile arrives by cp.async one tile ahead; one barrier per tile.  In
// the inner loop a thread's two field columns (both components, two 16-byte
// loads) feed all its rows, and each row's patterns are a broadcast load:
// 16 FMAs per row and sample.
#include "device.h"

namespace mlfma {

namespace {

__device__ __forceinline__ void cp16r(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void commit_r() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void wait_all_r() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// acc (two complex columns) += conj(v) * g
__device__ __forceinline__ void cmacc2(float4 &acc, float2 v, float4 g)
{
    acc.x = fmaf(v.x, g.x, fmaf(v.y, g.y, acc.x));
    acc.y = fmaf(v.x, g.y, fmaf(-v.y, g.x, acc.y));
    acc.z = fmaf(v.x, g.z, fmaf(v.y, g.w, acc.z));
    acc.w = fmaf(v.x, g.w, fmaf(-v.y, g.z, acc.w));
}

constexpr int kQT = 16;

template <int NCP, int MAXR>
__global__ void __launch_bounds__(256) k_receive_pairs(const int32_t *__restrict__ box_ptr, const float4 *__restrict__ V4,
                                                       DevLevel<float> lf, float2 *__restrict__ yp, int B, int Bs)
{
    constexpr int NG = 256 / NCP, NB = 2 * NCP, RCAP = NG * MAXR;
    constexpr int GT = 2 * kQT * NCP;   // float4 per field tile: [component][sample][column pair]
    constexpr int EPT = GT / 256;       // field elements staged per thread
    static_assert(GT % 256 == 0, "whole field tiles per thread");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4 *Gs = reinterpret_cast<float4 *>(smem_raw);   // [2][GT]
    float4 *Vs = Gs + 2 * GT;                            // [2][RCAP][kQT]
    const int K = lf.K;
    const int nch = (B + NB - 1) / NB, box = blockIdx.x / nch, b0 = (blockIdx.x - box * nch) * NB;
    const int nb = min(NB, B - b0);
    const int cp = threadIdx.x % NCP, grp = threadIdx.x / NCP;
    const int cols = 2 * cp + 1 < nb ? 2 : (2 * cp < nb ? 1 : 0);
    const bool a16 = (Bs % 2) == 0 && (B % 2) == 0 &&
                     ((reinterpret_cast<uintptr_t>(lf.G) | reinterpret_cast<uintptr_t>(yp)) & 15) == 0;
    const int i0 = box_ptr[box], nrows = box_ptr[box + 1] - i0;
    const float2 *G = reinterpret_cast<const float2 *>(lf.G) + (int64_t)box * 2 * K * Bs + b0 + 2 * cp;
    const float *wq = lf.wq;
    const int ntile = (K + kQT - 1) / kQT;
    // this thread's field elements: e = tid + k * 256 -> (component, sample, column pair = cp)
    auto load_g = [&](int tile, float4 (&g)[EPT]) {
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
            const int e = threadIdx.x + k * 256, m = e / (kQT * NCP), qx = (e / NCP) % kQT;
            const int q = tile * kQT + qx;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (q < K && cols) {
                const float2 *src = G + ((int64_t)m * K + q) * Bs;
                if (cols == 2 && a16) {
                    v = *reinterpret_cast<const float4 *>(src);
                } else {
                    const float2 a = src[0], b = cols == 2 ? src[1] : make_float2(0.f, 0.f);
                    v = make_float4(a.x, a.y, b.x, b.y);
                }
                const float w = wq[q];
                v.x *= w; v.y *= w; v.z *= w; v.w *= w;
            }
            g[k] = v;
        }
    };
    auto store_g = [&](int buf, const float4 (&g)[EPT]) {
#pragma unroll
        for (int k = 0; k < EPT; ++k) Gs[buf * GT + threadIdx.x + k * 256] = g[k];
    };
    for (int r0 = 0; r0 < nrows; r0 += RCAP) {
        const int nr = min(RCAP, nrows - r0);
        auto stage_v = [&](int tile, int buf) {
            const int q0 = tile * kQT;
            for (int e = threadIdx.x; e < nr * kQT; e += blockDim.x) {
                const int r = e / kQT, qx = e - r * kQT;
                float4 *d = Vs + ((size_t)buf * RCAP + r) * kQT + qx;
                if (q0 + qx < K) cp16r(d, V4 + (int64_t)(i0 + r0 + r) * K + q0 + qx);
                else *d = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            commit_r();
        };
        float4 acc[MAXR];
#pragma unroll
        for (int k = 0; k < MAXR; ++k) acc[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        {
            float4 g[EPT];
            load_g(0, g);
            stage_v(0, 0);
            store_g(0, g);
            wait_all_r();
            __syncthreads();
        }
        for (int tile = 0; tile < ntile; ++tile) {
            const int buf = tile & 1;
            float4 g[EPT];
            if (tile + 1 < ntile) {
                stage_v(tile + 1, buf ^ 1);
                load_g(tile + 1, g);
            }
            const float4 *gs = Gs + buf * GT + cp;
            const float4 *vs = Vs + (size_t)buf * RCAP * kQT;
#pragma unroll 4
            for (int qx = 0; qx < kQT; ++qx) {
                const float4 g0 = gs[qx * NCP], g1 = gs[(kQT + qx) * NCP];
#pragma unroll
                for (int k = 0; k < MAXR; ++k) {
                    const int r = grp + k * NG;
                    if (r < nr) {
                        const float4 v = vs[r * kQT + qx];
                        cmacc2(acc[k], make_float2(v.x, v.y), g0);
                        cmacc2(acc[k], make_float2(v.z, v.w), g1);
                    }
                }
            }
            if (tile + 1 < ntile) store_g(buf ^ 1, g);
            wait_all_r();
            __syncthreads();
        }
        if (cols) {
#pragma unroll
            for (int k = 0; k < MAXR; ++k) {
                const int r = grp + k * NG;
                if (r < nr) {
                    float2 *y = yp + (int64_t)(i0 + r0 + r) * B + b0 + 2 * cp;
                    const float4 a = acc[k];
                    if (cols == 2 && a16) {
                        float4 o = *reinterpret_cast<float4 *>(y);
                        o.x += a.x; o.y += a.y; o.z += a.z; o.w += a.w;
                        *reinterpret_cast<float4 *>(y) = o;
                    } else {
                        y[0] = make_float2(y[0].x + a.x, y[0].y + a.y);
                        if (cols == 2) y[1] = make_float2(y[1].x + a.z, y[1].y + a.w);
                    }
                }
            }
        }
    }
}

template <int NCP, int MAXR>
cudaError_t receive_pairs_nb(const ProductArgs<float> &a, int Bs, cudaStream_t s)
{
    constexpr int NG = 256 / NCP, RCAP = NG * MAXR, NB = 2 * NCP;
    const DevLevel<float> &Lf = a.lv[a.leaf];
    const size_t smem = ((size_t)2 * 2 * kQT * NCP + (size_t)2 * RCAP * kQT) * sizeof(float4);
    dim3 grid(Lf.nbox * ((a.B + NB - 1) / NB));
    k_receive_pairs<NCP, MAXR><<<grid, 256, smem, s>>>(a.nr.box_ptr, reinterpret_cast<const float4 *>(a.V), Lf,
                                                       reinterpret_cast<float2 *>(a.yp), a.B, Bs);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_receive_pairs(const ProductArgs<float> &a, int Bs, int nb, cudaStream_t s)
{
    switch (nb) {
    case 64: return receive_pairs_nb<32, 4>(a, Bs, s);
    case 32: return receive_pairs_nb<16, 2>(a, Bs, s);
    case 16: return receive_pairs_nb<8, 2>(a, Bs, s);
    default: return cudaErrorInvalidConfiguration;
    }
}

cudaError_t prime_receive_pairs()
{
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_receive_pairs<32, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_receive_pairs<16, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_receive_pairs<8, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
}

}  // namespace mlfma
