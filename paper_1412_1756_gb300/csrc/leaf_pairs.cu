// Radiation and reception of FP32 fields at the leaf level (Section III:
// the aggregation S_m(q) = sum_i V_i(q) x_i over the unknowns i of leaf box
// m, and the disaggregation y_i += sum_q w_q conj(V_i(q)) . G_m(q) over the
// samples q, both tangential components; w_q carries the quadrature weight
// and the far constant).
//
// Radiation: one CTA per (leaf box, chunk of 64 columns), 256 threads:
// thread = (four adjacent columns, two samples).  The box's x rows are staged
// once; the patterns stream through shared memory in steps of (32 samples,
// 32 rows) by cp.async one step ahead, one barrier per step.  Per row a
// thread's x quad (one 16-byte load) feeds both samples and both components:
// 32 FMAs per three 16-byte loads.
//
// Reception:
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

constexpr int kRQ = 32;   // samples per radiation step
constexpr int kRR = 32;   // rows per radiation step

__global__ void __launch_bounds__(256) k_radiate_quads(const int32_t *__restrict__ box_ptr, const float4 *__restrict__ V4,
                                                       const float *__restrict__ xp, float2 *__restrict__ S, int K,
                                                       int B, int Bs)
{
    constexpr int NQD = 16, NB = 4 * NQD;   // column quads, columns per CTA
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4 *Vs = reinterpret_cast<float4 *>(smem_raw);   // [2][kRR][kRQ]
    float4 *xs = Vs + 2 * kRR * kRQ;                     // [rows][NQD] (x of the box, four columns per float4)
    const int nch = (B + NB - 1) / NB, box = blockIdx.x / nch, b0 = (blockIdx.x - box * nch) * NB;
    const int nb = min(NB, B - b0);
    const int qd = threadIdx.x % NQD, ql = threadIdx.x / NQD;   // samples ql and ql + 16 of a step
    const int cols = max(0, min(4, nb - 4 * qd));
    const int j0 = box_ptr[box], nj = box_ptr[box + 1] - j0;
    const bool a16 = (B % 4) == 0 && (Bs % 2) == 0 &&
                     ((reinterpret_cast<uintptr_t>(xp) | reinterpret_cast<uintptr_t>(S)) & 15) == 0;
    // x rows of the box (zero past the chunk's columns)
    for (int e = threadIdx.x; e < nj * NQD; e += blockDim.x) {
        const int j = e / NQD, d = e - j * NQD, c = max(0, min(4, nb - 4 * d));
        const float *src = xp + (int64_t)(j0 + j) * B + b0 + 4 * d;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (c == 4 && a16) v = *reinterpret_cast<const float4 *>(src);
        else {
            if (c > 0) v.x = src[0];
            if (c > 1) v.y = src[1];
            if (c > 2) v.z = src[2];
            if (c > 3) v.w = src[3];
        }
        xs[e] = v;
    }
    const int ntile = (K + kRQ - 1) / kRQ, nchk = max(1, (nj + kRR - 1) / kRR), nstep = ntile * nchk;
    auto stage = [&](int step) {
        const int tile = step / nchk, chk = step - tile * nchk;
        const int q0 = tile * kRQ, r0 = chk * kRR, nr = min(kRR, nj - r0);
        float4 *d = Vs + (step & 1) * kRR * kRQ;
        for (int e = threadIdx.x; e < kRR * kRQ; e += blockDim.x) {
            const int r = e / kRQ, qx = e - r * kRQ;
            if (r < nr && q0 + qx < K) cp16r(d + e, V4 + (int64_t)(j0 + r0 + r) * K + q0 + qx);
            else d[e] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        commit_r();
    };
    float4 acc[2][2][2];   // [sample][component] (four columns as two float4 of complex pairs)
    auto zero = [&]() {
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int m = 0; m < 2; ++m) acc[a][m][0] = acc[a][m][1] = make_float4(0.f, 0.f, 0.f, 0.f);
    };
    zero();
    stage(0);
    for (int step = 0; step < nstep; ++step) {
        wait_all_r();
        __syncthreads();   // step's patterns in; everyone is done with the other buffer
        if (step + 1 < nstep) stage(step + 1);
        const int tile = step / nchk, chk = step - tile * nchk;
        const int r0 = chk * kRR, nr = min(kRR, nj - r0);
        const float4 *vs = Vs + (step & 1) * kRR * kRQ;
        const float4 *xr = xs + r0 * NQD + qd;
#pragma unroll 4
        for (int r = 0; r < nr; ++r) {
            const float4 x = xr[r * NQD];
            const float4 va = vs[r * kRQ + ql], vb = vs[r * kRQ + ql + 16];
            const float xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int s2 = 0; s2 < 2; ++s2) {
                const float4 v = s2 ? vb : va;   // (theta re, im, phi re, im) of the row at this sample
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    float4 &a0 = acc[s2][0][h], &a1 = acc[s2][1][h];
                    a0.x = fmaf(v.x, xv[2 * h], a0.x);
                    a0.y = fmaf(v.y, xv[2 * h], a0.y);
                    a0.z = fmaf(v.x, xv[2 * h + 1], a0.z);
                    a0.w = fmaf(v.y, xv[2 * h + 1], a0.w);
                    a1.x = fmaf(v.z, xv[2 * h], a1.x);
                    a1.y = fmaf(v.w, xv[2 * h], a1.y);
                    a1.z = fmaf(v.z, xv[2 * h + 1], a1.z);
                    a1.w = fmaf(v.w, xv[2 * h + 1], a1.w);
                }
            }
        }
        if (chk == nchk - 1) {   // the tile's sums are complete: store and restart
#pragma unroll
            for (int s2 = 0; s2 < 2; ++s2) {
                const int q = tile * kRQ + ql + 16 * s2;
                if (q < K && cols) {
#pragma unroll
                    for (int m = 0; m < 2; ++m) {
                        float2 *o = S + (((int64_t)box * 2 + m) * K + q) * Bs + b0 + 4 * qd;
                        if (cols == 4 && a16) {
                            reinterpret_cast<float4 *>(o)[0] = acc[s2][m][0];
                            reinterpret_cast<float4 *>(o)[1] = acc[s2][m][1];
                        } else {
                            const float2 v4[4] = {make_float2(acc[s2][m][0].x, acc[s2][m][0].y),
                                                  make_float2(acc[s2][m][0].z, acc[s2][m][0].w),
                                                  make_float2(acc[s2][m][1].x, acc[s2][m][1].y),
                                                  make_float2(acc[s2][m][1].z, acc[s2][m][1].w)};
#pragma unroll
                            for (int k = 0; k < 4; ++k)
                                if (k < cols) o[k] = v4[k];
                        }
                    }
                }
            }
            zero();
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

cudaError_t launch_radiate_quads(const ProductArgs<float> &a, int Bs, cudaStream_t s)
{
    const DevLevel<float> &Lf = a.lv[a.leaf];
    const size_t smem = ((size_t)2 * kRR * kRQ + (size_t)a.nr.max_rows * 16) * sizeof(float4);
    if (smem > (size_t)(96 * 1024)) return cudaErrorInvalidConfiguration;
    dim3 grid(Lf.nbox * ((a.B + 63) / 64));
    k_radiate_quads<<<grid, 256, smem, s>>>(a.nr.box_ptr, reinterpret_cast<const float4 *>(a.V), a.xp,
                                            reinterpret_cast<float2 *>(Lf.S), Lf.K, a.B, Bs);
    return cudaGetLastError();
}

cudaError_t prime_receive_pairs()
{
    if (cudaError_t e0 = cudaFuncSetAttribute(k_radiate_quads, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024))
        return e0;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_receive_pairs<32, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_receive_pairs<16, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_receive_pairs<8, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
}

}  // namespace mlfma
