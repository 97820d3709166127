// The multilevel fast multipole product y = Z x (Section III, Eq. (ZI)) as a
// chain of kernels, each templated on the real type R (float or double):
//
//   prepare    x (caller order) -> xp (leaf order, real columns)
//   near       y = Z_near x                       first term of Eq. (ZI)
//   radiate    S_m = sum_j V_s,mj x_j             aggregation, leaf level
//   up         S_p = sum_c shift_pc Interp(S_c)   (Section III-C)
//   translate  G_m = sum_{m' in IL(m)} alpha_mm' S_m'       (Eq. (8))
//   down       G_c += Anterp(conj(shift_pc) G_p)  (Section III-C)
//   receive    y_i += (-k^2 eta / 4 pi) sum_q w_q conj(V_s,mi) . G_m
//   finalize   y (leaf order, complex columns) -> caller order and type
//
// Fields are [box][component theta/phi][sample q][column b], b innermost,
// q theta-major.  Every kernel is memory- or latency-bound CUDA-core code:
// translation is diagonal in the samples and the local interpolation is
// banded, so neither is a dense contraction.  Data reuse is arranged in
// shared memory: the gathered x block of a near strip, a leaf box's x or G
// block, a child's field through both interpolation steps, and in the
// translation one source field applied to all children of a parent.
#include "device.h"

#include <algorithm>

namespace mlfma {

namespace {

template <class R> struct Cx;
template <> struct Cx<float> { using T = float2; using T4 = float4; };
template <> struct Cx<double> { using T = double2; using T4 = double4_32a; };

template <class C> __device__ __forceinline__ void cfma(C &acc, C a, C b)
{
    acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}
// acc += conj(a) * b
template <class C> __device__ __forceinline__ void cfmac(C &acc, C a, C b)
{
    acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(-a.y, b.x, acc.y));
}
template <class C, class R> __device__ __forceinline__ void rfma(C &acc, R s, C b)
{
    acc.x = fma(s, b.x, acc.x);
    acc.y = fma(s, b.y, acc.y);
}

// Asynchronous global -> shared copies of one complex value (8 or 16 bytes),
// completed by cp_async_wait: the copy's latency overlaps later work.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
template <class C>
__device__ __forceinline__ void cp_async(C *smem, const C *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (sizeof(C) == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

constexpr int kSmemCap = 227 * 1024;  // shared memory a CTA may use on sm_103a (static and dynamic together)
constexpr int kStageCap = 96 * 1024;  // staging budget of the near / leaf kernels (keeps >= 2 CTAs per SM)

inline int blocks_for(int64_t total, int threads)
{
    int64_t b = (total + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 64));
}

#define GRID_STRIDE(idx, total) \
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (total); idx += (int64_t)gridDim.x * blockDim.x)

// Lets `kernel` ask for the CTA's whole shared memory (the device's opt-in
// limit, at most kSmemCap) less what it declares statically.
template <class K>
cudaError_t allow_smem(K kernel)
{
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    const int cap = std::min(kSmemCap, optin) - (int)fa.sharedSizeBytes;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
}

// ------------------------------------------------------------ prepare ---
template <class R>
__global__ void k_prepare(const R *__restrict__ x, int xc, int Bu, int Bi, const int64_t *__restrict__ perm,
                          int64_t n, int adjoint, R *__restrict__ xp)
{
    GRID_STRIDE(idx, n * Bi)
    {
        const int64_t i = idx / Bi;
        const int b = (int)(idx % Bi);
        const int64_t src = perm[i];
        R v;
        if (!xc) {
            v = x[src * Bu + b];
        } else {
            const int part = b & 1;
            v = x[(src * Bu + (b >> 1)) * 2 + part];
            if (adjoint && part) v = -v;
        }
        xp[idx] = v;
    }
}

// ----------------------------------------------------------- finalize ---
template <class R>
__global__ void k_finalize(const typename Cx<R>::T *__restrict__ yp, int xc, int Bu, int Bi,
                           const int64_t *__restrict__ perm, int64_t n, int adjoint,
                           typename Cx<R>::T *__restrict__ y)
{
    using C = typename Cx<R>::T;
    GRID_STRIDE(idx, n * Bu)
    {
        const int64_t i = idx / Bu;
        const int b = (int)(idx % Bu);
        C v;
        if (!xc) {
            v = yp[i * Bi + b];
        } else {
            const C a = yp[i * Bi + 2 * b], c = yp[i * Bi + 2 * b + 1];
            v = C{a.x - c.y, a.y + c.x};   // Z x_r + i Z x_i
        }
        if (adjoint) v.y = -v.y;
        y[perm[i] * Bu + b] = v;
    }
}

// --------------------------------------------------------------- near ---
// One CTA per (leaf box, group of BT columns).  The box's strip [rows x
// neighbour columns] is column-major, so threads (g, r) walking columns
// c = g, g + G, ... read consecutive addresses; the gathered x block sits in
// shared memory (STAGE) when it fits.  Partial sums over g meet in shared
// memory.
template <class R, int BT, bool STAGE>
__global__ void __launch_bounds__(256) k_near(DevNear nr, const typename Cx<R>::T *__restrict__ val,
                                              const R *__restrict__ xp, typename Cx<R>::T *__restrict__ yp, int B)
{
    using C = typename Cx<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *xs = reinterpret_cast<R *>(smem_raw);
    __shared__ C red[256];
    // column chunk fastest in the grid: the CTAs that share a row's DRAM lines run together
    const int nch = (B + BT - 1) / BT, box = blockIdx.x / nch;
    const int b0 = (blockIdx.x - box * nch) * BT;
    const int nb = min(BT, B - b0);
    const int r0 = nr.box_ptr[box];
    const int nrow = nr.box_ptr[box + 1] - r0;
    const int c0 = nr.col_ptr[box];
    const int ncol = nr.col_ptr[box + 1] - c0;
    const int64_t off = nr.strip_off[box];
    const int t = threadIdx.x;
    if (STAGE) {
        for (int c = t; c < ncol; c += blockDim.x) {
            const R *xr = xp + (int64_t)nr.strip_col[c0 + c] * B + b0;
#pragma unroll
            for (int bb = 0; bb < BT; ++bb) xs[c * BT + bb] = bb < nb ? xr[bb] : R(0);
        }
        __syncthreads();
    }
    for (int rt = 0; rt < nrow; rt += blockDim.x) {
        const int RT = min(nrow - rt, (int)blockDim.x);
        const int G = blockDim.x / RT;
        const int r = t % RT, g = t / RT;
        const bool active = g < G;
        C acc[BT];
#pragma unroll
        for (int bb = 0; bb < BT; ++bb) acc[bb] = C{0, 0};
        if (active) {
            const C *v = val + off + rt + r;
            auto xcol = [&](int c, int bb) -> R {
                if (STAGE) return xs[c * BT + bb];
                return bb < nb ? xp[(int64_t)nr.strip_col[c0 + c] * B + b0 + bb] : R(0);
            };
            int c = g;
            for (; c + 3 * G < ncol; c += 4 * G) {
                const C z0 = v[(int64_t)c * nrow], z1 = v[(int64_t)(c + G) * nrow];
                const C z2 = v[(int64_t)(c + 2 * G) * nrow], z3 = v[(int64_t)(c + 3 * G) * nrow];
#pragma unroll
                for (int bb = 0; bb < BT; ++bb) {
                    rfma(acc[bb], xcol(c, bb), z0);
                    rfma(acc[bb], xcol(c + G, bb), z1);
                    rfma(acc[bb], xcol(c + 2 * G, bb), z2);
                    rfma(acc[bb], xcol(c + 3 * G, bb), z3);
                }
            }
            for (; c < ncol; c += G) {
                const C z = v[(int64_t)c * nrow];
#pragma unroll
                for (int bb = 0; bb < BT; ++bb) rfma(acc[bb], xcol(c, bb), z);
            }
        }
#pragma unroll
        for (int bb = 0; bb < BT; ++bb) {
            red[t] = active ? acc[bb] : C{0, 0};
            __syncthreads();
            if (t < RT && bb < nb) {
                C s{0, 0};
                for (int gg = 0; gg < G; ++gg) {
                    const C w = red[gg * RT + t];
                    s.x += w.x;
                    s.y += w.y;
                }
                yp[(int64_t)(r0 + rt + t) * B + b0 + bb] = s;
            }
            __syncthreads();
        }
    }
}

// Many columns: one CTA per leaf box and all B columns, so the strip is read
// from memory once.  Chunks of CCH strip columns - their values (contiguous
// in the column-major strip) and the x rows they multiply - are staged in
// shared memory by double-buffered asynchronous copies, so the next chunk's
// loads are in flight while this one is used; thread (row r, column group
// g) accumulates BPT columns of its row, its x values coming from one
// broadcast 16-byte load per 4 (FP32) or 2 (FP64) columns.  Needs B a
// multiple of 16 bytes of R; shared memory 2 CCH (B R + max_rows C).
template <class R, int BPT>
__global__ void __launch_bounds__(256) k_near_wide(DevNear nr, const typename Cx<R>::T *__restrict__ val,
                                                   const R *__restrict__ xp, typename Cx<R>::T *__restrict__ yp, int B)
{
    using C = typename Cx<R>::T;
    constexpr int CCH = 32;
    constexpr int VEC = 16 / sizeof(R);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *xs = reinterpret_cast<R *>(smem_raw);                       // [2][CCH][B]
    C *zs = reinterpret_cast<C *>(xs + (size_t)2 * CCH * B);       // [2][CCH][max_rows]
    const int box = blockIdx.x;
    const int r0 = nr.box_ptr[box];
    const int nrow = nr.box_ptr[box + 1] - r0;
    const int c0 = nr.col_ptr[box];
    const int ncol = nr.col_ptr[box + 1] - c0;
    const int64_t off = nr.strip_off[box];
    const int ng = (B + BPT - 1) / BPT;
    const int RT = max(1, min(nrow, (int)blockDim.x / ng));
    const int t = threadIdx.x, r = t % RT, g = t / RT;
    const bool active = g < ng;
    const int nchunk = (ncol + CCH - 1) / CCH;
    const int per = B / VEC;
    const int zpitch = nr.max_rows;
    auto stage = [&](int k) {
        const int cb = k * CCH, cn = min(CCH, ncol - cb);
        R *dst = xs + (size_t)(k & 1) * CCH * B;
        for (int e = t; e < cn * per; e += blockDim.x) {
            const int cc = e / per, p = e - cc * per;
            cp_async16(dst + cc * B + p * VEC, xp + (int64_t)nr.strip_col[c0 + cb + cc] * B + p * VEC);
        }
        C *zd = zs + (size_t)(k & 1) * CCH * zpitch;
        const C *zsrc = val + off + (int64_t)cb * nrow;
        for (int e = t; e < cn * nrow; e += blockDim.x) {
            const int cc = e / nrow, rr = e - cc * nrow;
            cp_async(zd + cc * zpitch + rr, zsrc + e);
        }
        cp_async_commit();
    };
    for (int rt = 0; rt < nrow; rt += RT) {
        C acc[BPT];
#pragma unroll
        for (int bb = 0; bb < BPT; ++bb) acc[bb] = C{0, 0};
        const bool live = active && rt + r < nrow;
        stage(0);
        for (int k = 0; k < nchunk; ++k) {
            if (k + 1 < nchunk) {
                stage(k + 1);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncthreads();
            if (live) {
                const R *xb = xs + (size_t)(k & 1) * CCH * B + g * BPT;
                const C *v = zs + (size_t)(k & 1) * CCH * zpitch + rt + r;
                const int cn = min(CCH, ncol - k * CCH);
#pragma unroll 4
                for (int cc = 0; cc < cn; ++cc) {
                    const C z = v[cc * zpitch];
                    const R *xr = xb + cc * B;
#pragma unroll
                    for (int bb = 0; bb < BPT; bb += VEC) {
                        if constexpr (VEC == 4) {
                            const float4 x4 = *reinterpret_cast<const float4 *>(xr + bb);
                            rfma(acc[bb], x4.x, z);
                            rfma(acc[bb + 1], x4.y, z);
                            rfma(acc[bb + 2], x4.z, z);
                            rfma(acc[bb + 3], x4.w, z);
                        } else {
                            const double2 x2 = *reinterpret_cast<const double2 *>(xr + bb);
                            rfma(acc[bb], x2.x, z);
                            rfma(acc[bb + 1], x2.y, z);
                        }
                    }
                }
            }
            __syncthreads();
        }
        if (live) {
            C *yr = yp + (int64_t)(r0 + rt + r) * B + g * BPT;
#pragma unroll
            for (int bb = 0; bb < BPT; ++bb)
                if (g * BPT + bb < B) yr[bb] = acc[bb];
        }
    }
}

// ------------------------------------------------------------ radiate ---
// S_m(q) = sum_{j in m} V_s,mj(q) x_j for one leaf box and a chunk of
// columns; both components from one 2-complex load; x block in shared memory.
template <class R>
__global__ void __launch_bounds__(256) k_radiate(const int32_t *__restrict__ box_ptr,
                                                 const typename Cx<R>::T4 *__restrict__ V4,
                                                 const R *__restrict__ xp, typename Cx<R>::T *__restrict__ S,
                                                 int K, int B, int Bt, int Bs)
{
    using C = typename Cx<R>::T;
    using C4 = typename Cx<R>::T4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *xs = reinterpret_cast<R *>(smem_raw);
    // column chunk fastest in the grid: the CTAs that share a row's DRAM lines run together
    const int nch = (B + Bt - 1) / Bt, box = blockIdx.x / nch;
    const int b0 = (blockIdx.x - box * nch) * Bt;
    const int nb = min(Bt, B - b0);
    const int j0 = box_ptr[box], nj = box_ptr[box + 1] - j0;
    for (int e = threadIdx.x; e < nj * nb; e += blockDim.x)
        xs[e] = xp[(int64_t)(j0 + e / nb) * B + b0 + e % nb];
    __syncthreads();
    for (int t = threadIdx.x; t < K * nb; t += blockDim.x) {
        const int q = t / nb, bb = t % nb;
        const C4 *vq = V4 + (int64_t)j0 * K + q;
        C a0{0, 0}, a1{0, 0};
        int j = 0;
        for (; j + 3 < nj; j += 4) {
            const C4 v0 = vq[(int64_t)j * K], v1 = vq[(int64_t)(j + 1) * K];
            const C4 v2 = vq[(int64_t)(j + 2) * K], v3 = vq[(int64_t)(j + 3) * K];
            const R x0 = xs[j * nb + bb], x1 = xs[(j + 1) * nb + bb], x2 = xs[(j + 2) * nb + bb],
                    x3 = xs[(j + 3) * nb + bb];
            a0.x = fma(v0.x, x0, fma(v1.x, x1, fma(v2.x, x2, fma(v3.x, x3, a0.x))));
            a0.y = fma(v0.y, x0, fma(v1.y, x1, fma(v2.y, x2, fma(v3.y, x3, a0.y))));
            a1.x = fma(v0.z, x0, fma(v1.z, x1, fma(v2.z, x2, fma(v3.z, x3, a1.x))));
            a1.y = fma(v0.w, x0, fma(v1.w, x1, fma(v2.w, x2, fma(v3.w, x3, a1.y))));
        }
        for (; j < nj; ++j) {
            const C4 v = vq[(int64_t)j * K];
            const R xv = xs[j * nb + bb];
            a0.x = fma(v.x, xv, a0.x);
            a0.y = fma(v.y, xv, a0.y);
            a1.x = fma(v.z, xv, a1.x);
            a1.y = fma(v.w, xv, a1.y);
        }
        S[((int64_t)(box * 2 + 0) * K + q) * Bs + b0 + bb] = a0;
        S[((int64_t)(box * 2 + 1) * K + q) * Bs + b0 + bb] = a1;
    }
}

// ---------------------------------------------------------- translate ---
// Eq. (8) sample by sample, grouped by parent: the children of one parent
// draw on one candidate set (children of the parent's neighbours), so each
// source field value is loaded once and applied to every child whose
// interaction list holds it.  A thread computes CB adjacent columns of one
// sample (one alpha load feeds CB columns); ES consecutive lanes may split
// the source list of one output and meet in a shuffle reduction (when a
// level has too few outputs to fill the GPU).  All children's accumulators
// live in registers.  With SA the CTA first copies the coefficients it
// needs - the parent's distinct translation types at the CTA's few samples -
// into shared memory, and the entries carry local type indices.
template <class R, int ES, int CB, bool SA>
__global__ void __launch_bounds__(128) k_translate(DevLevel<R> lv, int B, int Bs, int accumulate)
{
    using C = typename Cx<R>::T;
    __shared__ int s_src[216];
    __shared__ __align__(16) int16_t s_ty[216 * 8];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *s_al = reinterpret_cast<C *>(smem_raw);   // SA: [local type][NQ]
    const int P = blockIdx.x;
    const int e0 = lv.grp_ptr[P], ne = lv.grp_ptr[P + 1] - e0;
    const int m0 = lv.pchild_ptr[P], nc = lv.pchild_ptr[P + 1] - m0;
    const int K = lv.K;
    const int BC = B / CB;                 // column groups (B is a multiple of CB)
    const int outs = blockDim.x / ES;
    const int q_lo = (blockIdx.y * outs) / BC;
    const int NQ = min(K - 1, (blockIdx.y * outs + outs - 1) / BC) - q_lo + 1;
    if (SA) {
        const int l0 = lv.lty_ptr[P], nl = lv.lty_ptr[P + 1] - l0;
        const C *al = reinterpret_cast<const C *>(lv.alpha);
        for (int i = threadIdx.x; i < nl * NQ; i += blockDim.x) {
            const int lt = i / NQ, qq = i - lt * NQ;
            cp_async(s_al + i, al + (int64_t)lv.lty[l0 + lt] * K + q_lo + qq);
        }
        cp_async_commit();
    }
    const int16_t *tysrc = SA ? lv.grp_lty : lv.grp_ty;
    for (int e = threadIdx.x; e < ne; e += blockDim.x) s_src[e] = lv.grp_src[e0 + e];
    for (int e = threadIdx.x; e < ne * 8; e += blockDim.x) s_ty[e] = tysrc[(int64_t)e0 * 8 + e];
    if (SA) cp_async_wait<0>();
    __syncthreads();
    const int part = threadIdx.x % ES;
    const int t = blockIdx.y * outs + threadIdx.x / ES;
    const bool valid = t < K * BC;
    const int q = valid ? t / BC : 0, b = valid ? (t % BC) * CB : 0;
    const C *S = reinterpret_cast<const C *>(lv.S);
    const C *alpha = SA ? s_al + (q - q_lo) : reinterpret_cast<const C *>(lv.alpha) + q;
    const int astride = SA ? NQ : K;
    C acc[8][2][CB];
#pragma unroll
    for (int c = 0; c < 8; ++c)
#pragma unroll
        for (int k = 0; k < CB; ++k) acc[c][0][k] = acc[c][1][k] = C{0, 0};
    const int64_t KB = (int64_t)K * Bs;
    const int64_t qb = (int64_t)q * Bs + b;
    if (valid) {
#pragma unroll 2
        for (int e = part; e < ne; e += ES) {
            const int64_t base = (int64_t)s_src[e] * 2 * KB + qb;
            C s0[CB], s1[CB];
#pragma unroll
            for (int k = 0; k < CB; ++k) {
                s0[k] = S[base + k];
                s1[k] = S[base + KB + k];
            }
            const int4 tyv = *reinterpret_cast<const int4 *>(&s_ty[e * 8]);
            const int tw[4] = {tyv.x, tyv.y, tyv.z, tyv.w};
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                if (c >= nc) break;   // the parent's children occupy slots 0 .. nc-1
                const int ty = (int)(int16_t)((tw[c >> 1] >> (16 * (c & 1))) & 0xffff);
                if (ty >= 0) {
                    const C al = alpha[ty * astride];
#pragma unroll
                    for (int k = 0; k < CB; ++k) {
                        cfma(acc[c][0][k], al, s0[k]);
                        cfma(acc[c][1][k], al, s1[k]);
                    }
                }
            }
        }
    }
    if (ES > 1) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            if (c >= nc) break;
#pragma unroll
            for (int off = ES / 2; off >= 1; off >>= 1)
#pragma unroll
                for (int m = 0; m < 2; ++m)
#pragma unroll
                    for (int k = 0; k < CB; ++k) {
                        acc[c][m][k].x += __shfl_xor_sync(0xffffffffu, acc[c][m][k].x, off);
                        acc[c][m][k].y += __shfl_xor_sync(0xffffffffu, acc[c][m][k].y, off);
                    }
        }
    }
    if (!valid || part != 0) return;
    C *G = reinterpret_cast<C *>(lv.G);
#pragma unroll
    for (int c = 0; c < 8; ++c)
        if (c < nc) {
            const int64_t o = (int64_t)(m0 + c) * 2 * KB + qb;
#pragma unroll
            for (int k = 0; k < CB; ++k) {
                if (accumulate) {
                    C g0 = G[o + k], g1 = G[o + KB + k];
                    g0.x += acc[c][0][k].x; g0.y += acc[c][0][k].y;
                    g1.x += acc[c][1][k].x; g1.y += acc[c][1][k].y;
                    G[o + k] = g0;
                    G[o + KB + k] = g1;
                } else {
                    G[o + k] = acc[c][0][k];
                    G[o + KB + k] = acc[c][1][k];
                }
            }
        }
}

// Translation, one warp per (child, sample): the child's own interaction
// list (no per-entry child decode), CB columns per lane and 32 CB columns
// per pass; a CTA covers one parent's children at QC samples, so the
// sources they share are read from memory once and from L1 afterwards.
// The coefficients of every type of the level at the CTA's samples are
// staged in shared memory.  A candidate of the autotuner.
template <class R, int CB, int QC>
__global__ void __launch_bounds__(256) k_translate_cw(DevLevel<R> lv, int B, int Bs, int accumulate)
{
    using C = typename Cx<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *s_al = reinterpret_cast<C *>(smem_raw);   // [type][QC]
    const int P = blockIdx.x, q0 = blockIdx.y * QC, K = lv.K;
    const int nq = min(QC, K - q0);
    const int m0 = lv.pchild_ptr[P], nc = lv.pchild_ptr[P + 1] - m0;
    const C *al = reinterpret_cast<const C *>(lv.alpha);
    for (int i = threadIdx.x; i < lv.ntype * QC; i += blockDim.x) {
        const int ty = i / QC, qq = i - ty * QC;
        if (qq < nq) cp_async(s_al + i, al + (int64_t)ty * K + q0 + qq);
        else s_al[i] = C{0, 0};
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const C *S = reinterpret_cast<const C *>(lv.S);
    C *G = reinterpret_cast<C *>(lv.G);
    const int64_t KB = (int64_t)K * Bs;
    for (int pr = warp; pr < nc * QC; pr += blockDim.x >> 5) {
        const int c = pr / QC, qq = pr - c * QC;
        if (qq >= nq) continue;
        const int m = m0 + c, q = q0 + qq;
        const int e0 = lv.il_ptr[m], e1 = lv.il_ptr[m + 1];
        for (int bp = 0; bp < B; bp += 32 * CB) {
            const int b = bp + lane * CB;
            if (b >= B) break;
            C acc[2][CB];
#pragma unroll
            for (int k = 0; k < CB; ++k) acc[0][k] = acc[1][k] = C{0, 0};
#pragma unroll 4
            for (int e = e0; e < e1; ++e) {
                const int src = lv.il_src[e], ty = lv.il_type[e];
                const C a = s_al[ty * QC + qq];
                const int64_t base = (int64_t)src * 2 * KB + (int64_t)q * Bs + b;
#pragma unroll
                for (int k = 0; k < CB; ++k) {
                    if (b + k < B) {
                        cfma(acc[0][k], a, S[base + k]);
                        cfma(acc[1][k], a, S[base + KB + k]);
                    }
                }
            }
            const int64_t o = (int64_t)m * 2 * KB + (int64_t)q * Bs + b;
#pragma unroll
            for (int k = 0; k < CB; ++k) {
                if (b + k >= B) break;
                if (accumulate) {
                    C g0 = G[o + k], g1 = G[o + KB + k];
                    g0.x += acc[0][k].x; g0.y += acc[0][k].y;
                    g1.x += acc[1][k].x; g1.y += acc[1][k].y;
                    G[o + k] = g0;
                    G[o + KB + k] = g1;
                } else {
                    G[o + k] = acc[0][k];
                    G[o + KB + k] = acc[1][k];
                }
            }
        }
    }
}

// ----------------------------------------------------------- upward ---
// CP adjacent columns per thread (2 for FP32: one 16-byte shared-memory
// access moves both).
template <class R, int NB> struct ColPair { static constexpr int CP = (sizeof(R) == 4 && NB >= 2) ? 2 : 1; };

template <class C, int CP>
__device__ __forceinline__ void lds_cols(const C *p, C (&v)[CP])
{
    if constexpr (CP == 2) {
        const float4 q = *reinterpret_cast<const float4 *>(p);
        v[0] = C{q.x, q.y};
        v[1] = C{q.z, q.w};
    } else {
        v[0] = p[0];
    }
}
template <class C, int CP>
__device__ __forceinline__ void sts_cols(C *p, const C (&v)[CP])
{
    if constexpr (CP == 2) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
    } else {
        p[0] = v[0];
    }
}

// Work split of a stencil step: items are (stencil row `key`, column group)
// x chunks of the `span` rows the stencil row applies to; a thread loads an
// item's taps into registers once and sweeps the chunk.  Threads loop over
// items when there are more than the CTA has threads.
struct Split {
    int per, chunks, len, items;
    __device__ Split(int keys, int span, int NL)
    {
        per = keys * NL;
        chunks = max(1, (int)blockDim.x / per);
        len = (span + chunks - 1) / chunks;
        items = per * chunks;
    }
    __device__ void item(int it, int NL, int CP, int span, int &key, int &cg, int &lo, int &hi) const
    {
        key = (it % per) / NL;
        cg = (it % NL) * CP;
        lo = (it / per) * len;
        hi = min(span, lo + len);
    }
};

// Interleaved variant: item (key, column group, phase ch) takes the rows
// ch, ch + chunks, ...; the threads of a quarter warp then read adjacent
// rows of one key (bank-conflict free when rows are PW columns wide).
struct SplitIL {
    int chunks, items, NLc;
    __device__ SplitIL(int keys, int NL)
    {
        NLc = NL;
        chunks = max(1, (int)blockDim.x / (keys * NL));
        items = keys * NL * chunks;
    }
    __device__ void item(int it, int CP, int &key, int &cg, int &ch) const
    {
        cg = (it % NLc) * CP;
        ch = (it / NLc) % chunks;
        key = it / (NLc * chunks);
    }
};

// One CTA per (parent box, component, chunk of NB columns, band of parent
// theta rows).  Per child: its field -> shared memory (the next child's
// field is prefetched into registers meanwhile), theta interpolation of the
// band's rows -> shared memory, phi interpolation and phase shift
// accumulated into the band's outputs in shared memory; one store of the
// parent field at the end.  In each stencil step a thread holds the PO taps
// of one stencil row in registers and applies them to a chunk of rows.
// Parent theta rows per band of a CTA (even when the rows go in pairs).
__host__ __device__ inline int up_band_rows(int ntp, int RS, int RB)
{
    const int rows = (ntp + RS - 1) / RS;
    return RB == 2 ? rows + (rows & 1) : rows;
}

// RB = 2: the interpolation rows go in pairs (tables thu2 / phu2: the union of
// both rows' taps, PO entries, one coefficient per row), so each value a
// thread loads from shared memory feeds both rows of the pair.
template <class R, int NB, int PO, int RB = 1>
__global__ void __launch_bounds__(256) k_up(DevLevel<R> P, DevLevel<R> Ch, int B, int RS, int Bs, int accumulate)
{
    using C = typename Cx<R>::T;
    constexpr int CP = ColPair<R, NB>::CP, NL = NB / CP, PW = NB;
    constexpr int PF = 8;   // prefetch registers per thread
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Kc = Ch.K, nphc = Ch.nph, hc = nphc / 2, ntp = P.nth, nphp = P.nph;
    // column chunk fastest in the grid, then the band, then the parent
    const int comp = blockIdx.y;
    const int nbc = (B + NB - 1) / NB, p = blockIdx.x / (nbc * RS), rem = blockIdx.x - p * (nbc * RS);
    const int rs = rem / nbc, b0 = (rem - rs * nbc) * NB;
    const int rows = up_band_rows(ntp, RS, RB), t0 = rs * rows, t1 = min(ntp, t0 + rows);
    if (t0 >= t1) return;
    const int nr = t1 - t0;
    const int nb = min(NB, B - b0);
    const int bb = threadIdx.x % NB, slot = threadIdx.x / NB, nslot = blockDim.x / NB;
    const bool bok = bb < nb;
    const int nT = nr * nphc, nO = nr * nphp;
    C *A = reinterpret_cast<C *>(smem_raw);   // [Kc][NB]
    C *T = A + (size_t)Kc * PW;                // [nT][NB]
    C *O = T + (size_t)nT * PW;                // [nO][NB]
    const C *S = reinterpret_cast<const C *>(Ch.S);
    const C *shift = reinterpret_cast<const C *>(P.shift) + (int64_t)t0 * nphp;
    for (int e = threadIdx.x; e < nO * PW; e += blockDim.x) O[e] = C{0, 0};
    const SplitIL st((nr + RB - 1) / RB, NL);   // theta step: key = band theta row (pair), rows = child phi index
    const Split sp(nphp / RB, nr, NL);          // phi step: key = parent phi index (pair), span = band theta rows
    const int c0 = P.child_ptr[p], c1 = P.child_ptr[p + 1];
    C pre[PF];
    auto fetch = [&](int c) {
        const C *src = S + ((int64_t)c * 2 + comp) * Kc * Bs + b0 + bb;
#pragma unroll
        for (int k = 0; k < PF; ++k) {
            const int q = slot + k * nslot;
            pre[k] = (bok && q < Kc) ? src[(int64_t)q * Bs] : C{0, 0};
        }
    };
    fetch(c0);
    for (int c = c0; c < c1; ++c) {
#pragma unroll
        for (int k = 0; k < PF; ++k) {
            const int q = slot + k * nslot;
            if (q < Kc) A[q * PW + bb] = pre[k];
        }
        if (PF * nslot < Kc) {
            const C *src = S + ((int64_t)c * 2 + comp) * Kc * Bs + b0 + bb;
#pragma unroll 4
            for (int q = slot + PF * nslot; q < Kc; q += nslot) A[q * PW + bb] = bok ? src[(int64_t)q * Bs] : C{0, 0};
        }
        __syncthreads();
        if (c + 1 < c1) fetch(c + 1);
        for (int it = threadIdx.x; it < st.items; it += blockDim.x) {
            int key, cg, ch;
            st.item(it, CP, key, cg, ch);
            int tb[PO];
            bool rf[PO];
            R tc[RB][PO];
#pragma unroll
            for (int f = 0; f < PO; ++f) {
                int ti;
                if constexpr (RB == 1) {
                    const Tap<R> tap = P.thu[(size_t)(t0 + key) * PO + f];
                    ti = tap.i;
                    tc[0][f] = tap.c;
                } else {
                    const Tap2<R> tap = P.thu2[(size_t)(t0 / 2 + key) * PO + f];
                    ti = tap.i;
                    tc[0][f] = tap.c[0];
                    tc[1][f] = tap.c[1];
                }
                tb[f] = (ti & (kTapRefl - 1)) * nphc;
                rf[f] = (ti & kTapRefl) != 0;
            }
            for (int v = ch; v < nphc; v += st.chunks) {
                const int vs = v + hc < nphc ? v + hc : v + hc - nphc;
                C s[RB][CP];
#pragma unroll
                for (int r = 0; r < RB; ++r)
#pragma unroll
                    for (int k = 0; k < CP; ++k) s[r][k] = C{0, 0};
#pragma unroll
                for (int f = 0; f < PO; ++f) {
                    C a[CP];
                    lds_cols<C, CP>(A + (tb[f] + (rf[f] ? vs : v)) * PW + cg, a);
#pragma unroll
                    for (int r = 0; r < RB; ++r)
#pragma unroll
                        for (int k = 0; k < CP; ++k) rfma(s[r][k], tc[r][f], a[k]);
                }
#pragma unroll
                for (int r = 0; r < RB; ++r)
                    if (key * RB + r < nr) sts_cols<C, CP>(T + ((key * RB + r) * nphc + v) * PW + cg, s[r]);
            }
        }
        __syncthreads();
        const C *sh = shift + (int64_t)Ch.octant[c] * P.K;
        for (int it = threadIdx.x; it < sp.items; it += blockDim.x) {
            int key, cg, lo, hi;
            sp.item(it, NL, CP, nr, key, cg, lo, hi);
            int pb[PO];
            R pc[RB][PO];
#pragma unroll
            for (int f = 0; f < PO; ++f) {
                if constexpr (RB == 1) {
                    const Tap<R> tap = P.phu[(size_t)key * PO + f];
                    pb[f] = tap.i;
                    pc[0][f] = tap.c;
                } else {
                    const Tap2<R> tap = P.phu2[(size_t)key * PO + f];
                    pb[f] = tap.i;
                    pc[0][f] = tap.c[0];
                    pc[1][f] = tap.c[1];
                }
            }
            for (int tr = lo; tr < hi; ++tr) {
                const C *trow = T + tr * nphc * PW + cg;
                C s[RB][CP];
#pragma unroll
                for (int r = 0; r < RB; ++r)
#pragma unroll
                    for (int k = 0; k < CP; ++k) s[r][k] = C{0, 0};
#pragma unroll
                for (int f = 0; f < PO; ++f) {
                    C a[CP];
                    lds_cols<C, CP>(trow + pb[f] * PW, a);
#pragma unroll
                    for (int r = 0; r < RB; ++r)
#pragma unroll
                        for (int k = 0; k < CP; ++k) rfma(s[r][k], pc[r][f], a[k]);
                }
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    const int o = tr * nphp + key * RB + r;
                    const C z = sh[o];
                    C acc[CP];
                    lds_cols<C, CP>(O + o * PW + cg, acc);
#pragma unroll
                    for (int k = 0; k < CP; ++k) cfma(acc[k], z, s[r][k]);
                    sts_cols<C, CP>(O + o * PW + cg, acc);
                }
            }
        }
        __syncthreads();
    }
    if (!bok) return;
    C *dst = reinterpret_cast<C *>(P.S) + (((int64_t)p * 2 + comp) * P.K + (int64_t)t0 * nphp) * Bs + b0 + bb;
    if (accumulate) {
        for (int o = slot; o < nO; o += nslot) {
            C y = dst[(int64_t)o * Bs];
            const C d = O[o * PW + bb];
            y.x += d.x;
            y.y += d.y;
            dst[(int64_t)o * Bs] = y;
        }
    } else {
        for (int o = slot; o < nO; o += nslot) dst[(int64_t)o * Bs] = O[o * PW + bb];
    }
}

// --------------------------------------------------------- downward ---
// One CTA per (child box, component, chunk of NB columns).  At entry both the
// parent's incoming field and the child's own are requested with
// asynchronous copies into shared memory; the parent's is multiplied by the
// conjugate shift in place, phi anterpolation -> shared memory, theta
// anterpolation -> shared memory (over the first buffer), and the child's
// copy (waited for only now) plus the result is stored back.  The
// anterpolation stencils (weighted transposes of the interpolation
// stencils) are zero-padded to TM taps per row so that a thread holds one
// row's taps in registers and sweeps them over a chunk of rows, CP adjacent
// columns per 16-byte shared-memory access (the layout of the upward pass).
// RB = 2: the anterpolation rows go in pairs (tables thd2 / phd2: the union of
// both rows' taps, one coefficient per row), so each value a thread loads
// from shared memory feeds both rows of the pair.
template <class R, int NB, int TM, int RB = 1>
__global__ void __launch_bounds__(256, (sizeof(R) == 4 && TM <= 20) ? (RB == 1 ? 4 : (TM <= 16 ? 3 : 2)) : 1)
    k_down(DevLevel<R> P, DevLevel<R> Ch, int B, int Bs)
{
    using C = typename Cx<R>::T;
    constexpr int CP = ColPair<R, NB>::CP, NL = NB / CP, PW = NB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Kc = Ch.K, nthc = Ch.nth, nphc = Ch.nph, hc = nphc / 2, ntp = P.nth, nphp = P.nph, Kp = P.K;
    // column chunk fastest in the grid: the CTAs that share a row's DRAM lines run together
    const int nbc = (B + NB - 1) / NB, c = blockIdx.x / nbc, comp = blockIdx.y;
    const int b0 = (blockIdx.x - c * nbc) * NB;
    const int nb = min(NB, B - b0);
    const int hp = nphp + 1;                   // H row pitch per parent theta row (one pad row)
    C *H = reinterpret_cast<C *>(smem_raw);   // [ntp][hp][PW]; later the child result [Kc][PW]
    C *U = H + (size_t)ntp * hp * PW;          // [ntp * nphc][PW]
    C *X = U + (size_t)ntp * nphc * PW;        // [Kc][PW] the child's incoming field
    const int bb = threadIdx.x % NB, slot = threadIdx.x / NB, nslot = blockDim.x / NB;
    const bool bok = bb < nb;
    C *dst = reinterpret_cast<C *>(Ch.G) + ((int64_t)c * 2 + comp) * Kc * Bs + b0 + bb;
    {
        const int par = Ch.parent[c];
        const C *g = reinterpret_cast<const C *>(P.G) + ((int64_t)par * 2 + comp) * Kp * Bs + b0 + bb;
        for (int q = slot; q < Kp; q += nslot) {
            const int hq = q + q / nphp;   // padded row
            if (bok) cp_async(H + hq * PW + bb, g + (int64_t)q * Bs);
            else H[hq * PW + bb] = C{0, 0};
        }
        cp_async_commit();
        if (bok)
            for (int q = slot; q < Kc; q += nslot) cp_async(X + q * PW + bb, dst + (int64_t)q * Bs);
        cp_async_commit();
        const C *sh = reinterpret_cast<const C *>(P.shift) + (int64_t)Ch.octant[c] * Kp;
        cp_async_wait<1>();
#pragma unroll 4
        for (int q = slot; q < Kp; q += nslot) {   // the elements this thread copied
            const int hq = q + q / nphp;
            C h{0, 0};
            cfmac(h, sh[q], H[hq * PW + bb]);
            H[hq * PW + bb] = h;
        }
    }
    __syncthreads();
    // phi: U(tp, v) = sum_f c_f H(tp, u_f(v)); key = child phi index v (a pair
    // of them for RB = 2), rows = parent theta rows
    const SplitIL sp((nphc + RB - 1) / RB, NL);
    for (int it = threadIdx.x; it < sp.items; it += blockDim.x) {
        int key, cg, ch;
        sp.item(it, CP, key, cg, ch);
        int pb[TM];
        R pc[RB][TM];
#pragma unroll
        for (int f = 0; f < TM; ++f) {
            if constexpr (RB == 1) {
                const Tap<R> tap = P.phd_pad[(size_t)key * TM + f];
                pb[f] = tap.i * PW;
                pc[0][f] = tap.c;
            } else {
                const Tap2<R> tap = P.phd2[(size_t)key * TM + f];
                pb[f] = tap.i * PW;
                pc[0][f] = tap.c[0];
                pc[1][f] = tap.c[1];
            }
        }
        for (int tp = ch; tp < ntp; tp += sp.chunks) {
            const C *hrow = H + tp * hp * PW + cg;
            C s[RB][CP];
#pragma unroll
            for (int r = 0; r < RB; ++r)
#pragma unroll
                for (int k = 0; k < CP; ++k) s[r][k] = C{0, 0};
#pragma unroll
            for (int f = 0; f < TM; ++f) {
                C a[CP];
                lds_cols<C, CP>(hrow + pb[f], a);
#pragma unroll
                for (int r = 0; r < RB; ++r)
#pragma unroll
                    for (int k = 0; k < CP; ++k) rfma(s[r][k], pc[r][f], a[k]);
            }
#pragma unroll
            for (int r = 0; r < RB; ++r)
                if (key * RB + r < nphc) sts_cols<C, CP>(U + (tp * nphc + key * RB + r) * PW + cg, s[r]);
        }
    }
    __syncthreads();
    // theta: W(j, v) = sum_f c_f U(t_f, v or v + pi); key = child theta row j
    // (a pair of them for RB = 2), span = child phi index
    const SplitIL st((nthc + RB - 1) / RB, NL);
    C *W = H;
    for (int it = threadIdx.x; it < st.items; it += blockDim.x) {
        int key, cg, ch;
        st.item(it, CP, key, cg, ch);
        int tb[TM];
        bool rf[TM];
        R tc[RB][TM];
#pragma unroll
        for (int f = 0; f < TM; ++f) {
            int ti;
            if constexpr (RB == 1) {
                const Tap<R> tap = P.thd_pad[(size_t)key * TM + f];
                ti = tap.i;
                tc[0][f] = tap.c;
            } else {
                const Tap2<R> tap = P.thd2[(size_t)key * TM + f];
                ti = tap.i;
                tc[0][f] = tap.c[0];
                tc[1][f] = tap.c[1];
            }
            tb[f] = (ti & (kTapRefl - 1)) * nphc;
            rf[f] = (ti & kTapRefl) != 0;
        }
        for (int v = ch; v < nphc; v += st.chunks) {
            const int vs = v + hc < nphc ? v + hc : v + hc - nphc;
            C s[RB][CP];
#pragma unroll
            for (int r = 0; r < RB; ++r)
#pragma unroll
                for (int k = 0; k < CP; ++k) s[r][k] = C{0, 0};
#pragma unroll
            for (int f = 0; f < TM; ++f) {
                C a[CP];
                lds_cols<C, CP>(U + (tb[f] + (rf[f] ? vs : v)) * PW + cg, a);
#pragma unroll
                for (int r = 0; r < RB; ++r)
#pragma unroll
                    for (int k = 0; k < CP; ++k) rfma(s[r][k], tc[r][f], a[k]);
            }
#pragma unroll
            for (int r = 0; r < RB; ++r)
                if (key * RB + r < nthc) sts_cols<C, CP>(W + ((key * RB + r) * nphc + v) * PW + cg, s[r]);
        }
    }
    cp_async_wait<0>();
    __syncthreads();
    if (!bok) return;
#pragma unroll 8
    for (int q = slot; q < Kc; q += nslot) {   // X elements: copied by this thread
        C y = X[q * PW + bb];
        const C w = W[q * PW + bb];
        y.x += w.x;
        y.y += w.y;
        dst[(int64_t)q * Bs] = y;
    }
}

// Per parent: one CTA per (parent box, component, chunk of NB columns)
// loads the parent's incoming field once (cp.async) and loops over its
// children - conjugate shift into H, phi and theta anterpolation as in
// k_down, the child's own field prefetched during the stencil work - so
// the parent load and the CTA overheads are shared by the children.  A
// candidate of the autotuner.
template <class R, int NB, int TM>
__global__ void __launch_bounds__(256, (sizeof(R) == 4 && TM <= 20) ? 2 : 1)
    k_down_pp(DevLevel<R> P, DevLevel<R> Ch, int B, int Bs)
{
    using C = typename Cx<R>::T;
    constexpr int CP = ColPair<R, NB>::CP, NL = NB / CP, PW = NB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Kc = Ch.K, nthc = Ch.nth, nphc = Ch.nph, hc = nphc / 2, ntp = P.nth, nphp = P.nph, Kp = P.K;
    const int nbc = (B + NB - 1) / NB, p = blockIdx.x / nbc, comp = blockIdx.y, b0 = (blockIdx.x - p * nbc) * NB;
    const int nb = min(NB, B - b0);
    const int hp = nphp + 1;
    C *Gp = reinterpret_cast<C *>(smem_raw);   // [Kp][PW] the parent's field
    C *H = Gp + (size_t)Kp * PW;                // [ntp][hp][PW]; later the child result [Kc][PW]
    C *U = H + (size_t)ntp * hp * PW;          // [ntp * nphc][PW]
    C *X = U + (size_t)ntp * nphc * PW;        // [Kc][PW] the child's incoming field
    const int bb = threadIdx.x % NB, slot = threadIdx.x / NB, nslot = blockDim.x / NB;
    const bool bok = bb < nb;
    {
        const C *g = reinterpret_cast<const C *>(P.G) + ((int64_t)p * 2 + comp) * Kp * Bs + b0 + bb;
        for (int q = slot; q < Kp; q += nslot) {
            if (bok) cp_async(Gp + q * PW + bb, g + (int64_t)q * Bs);
            else Gp[q * PW + bb] = C{0, 0};
        }
        cp_async_commit();
    }
    const SplitIL sp(nphc, NL), st(nthc, NL);
    const int c0 = P.child_ptr[p], c1 = P.child_ptr[p + 1];
    for (int c = c0; c < c1; ++c) {
        C *dst = reinterpret_cast<C *>(Ch.G) + ((int64_t)c * 2 + comp) * Kc * Bs + b0 + bb;
        if (bok)
            for (int q = slot; q < Kc; q += nslot) cp_async(X + q * PW + bb, dst + (int64_t)q * Bs);
        cp_async_commit();
        cp_async_wait<1>();   // the parent's field (and any older group)
        __syncthreads();
        const C *sh = reinterpret_cast<const C *>(P.shift) + (int64_t)Ch.octant[c] * Kp;
#pragma unroll 4
        for (int q = slot; q < Kp; q += nslot) {
            C h{0, 0};
            cfmac(h, sh[q], Gp[q * PW + bb]);
            H[(q + q / nphp) * PW + bb] = h;
        }
        __syncthreads();
        for (int it = threadIdx.x; it < sp.items; it += blockDim.x) {
            int key, cg, ch;
            sp.item(it, CP, key, cg, ch);
            int pb[TM];
            R pc[TM];
#pragma unroll
            for (int f = 0; f < TM; ++f) {
                const Tap<R> tap = P.phd_pad[(size_t)key * TM + f];
                pb[f] = tap.i * PW;
                pc[f] = tap.c;
            }
            for (int tp = ch; tp < ntp; tp += sp.chunks) {
                const C *hrow = H + tp * hp * PW + cg;
                C s[CP];
#pragma unroll
                for (int k = 0; k < CP; ++k) s[k] = C{0, 0};
#pragma unroll
                for (int f = 0; f < TM; ++f) {
                    C a[CP];
                    lds_cols<C, CP>(hrow + pb[f], a);
#pragma unroll
                    for (int k = 0; k < CP; ++k) rfma(s[k], pc[f], a[k]);
                }
                sts_cols<C, CP>(U + (tp * nphc + key) * PW + cg, s);
            }
        }
        __syncthreads();
        C *W = H;
        for (int it = threadIdx.x; it < st.items; it += blockDim.x) {
            int key, cg, ch;
            st.item(it, CP, key, cg, ch);
            int tb[TM];
            bool rf[TM];
            R tc[TM];
#pragma unroll
            for (int f = 0; f < TM; ++f) {
                const Tap<R> tap = P.thd_pad[(size_t)key * TM + f];
                tb[f] = (tap.i & (kTapRefl - 1)) * nphc;
                rf[f] = (tap.i & kTapRefl) != 0;
                tc[f] = tap.c;
            }
            for (int v = ch; v < nphc; v += st.chunks) {
                const int vs = v + hc < nphc ? v + hc : v + hc - nphc;
                C s[CP];
#pragma unroll
                for (int k = 0; k < CP; ++k) s[k] = C{0, 0};
#pragma unroll
                for (int f = 0; f < TM; ++f) {
                    C a[CP];
                    lds_cols<C, CP>(U + (tb[f] + (rf[f] ? vs : v)) * PW + cg, a);
#pragma unroll
                    for (int k = 0; k < CP; ++k) rfma(s[k], tc[f], a[k]);
                }
                sts_cols<C, CP>(W + (key * nphc + v) * PW + cg, s);
            }
        }
        cp_async_wait<0>();
        __syncthreads();
        if (bok) {
#pragma unroll 8
            for (int q = slot; q < Kc; q += nslot) {
                C y = X[q * PW + bb];
                const C w = W[q * PW + bb];
                y.x += w.x;
                y.y += w.y;
                dst[(int64_t)q * Bs] = y;
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ receive ---
// y_i += sum_q wq_q conj(V_s,mi(q)) . G_m(q).
// Few columns: one CTA per (leaf box, chunk of LB columns) with the box's G
// block in shared memory; one warp per unknown at a time, lanes split into
// LB column lanes x 32/LB sample lanes, reduced with shuffles.
template <class R, int LB>
__global__ void __launch_bounds__(256) k_receive(const int32_t *__restrict__ box_ptr,
                                                 const typename Cx<R>::T4 *__restrict__ V4, DevLevel<R> lf,
                                                 typename Cx<R>::T *__restrict__ yp, int B, int Bs)
{
    using C = typename Cx<R>::T;
    using C4 = typename Cx<R>::T4;
    constexpr int LQ = 32 / LB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *Gs = reinterpret_cast<C *>(smem_raw);   // [2][K][LB]
    const int K = lf.K;
    // column chunk fastest in the grid: the CTAs that share a row's DRAM lines run together
    const int nch = (B + LB - 1) / LB, box = blockIdx.x / nch;
    const int b0 = (blockIdx.x - box * nch) * LB;
    const int nb = min(LB, B - b0);
    const C *G = reinterpret_cast<const C *>(lf.G) + (int64_t)box * 2 * K * Bs + b0;
    for (int e = threadIdx.x; e < 2 * K * LB; e += blockDim.x) {
        const int bb = e % LB;
        Gs[e] = bb < nb ? G[(int64_t)(e / LB) * Bs + bb] : C{0, 0};
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int lb = lane % LB, lq = lane / LB;
    const int i0 = box_ptr[box], i1 = box_ptr[box + 1];
    for (int i = i0 + warp; i < i1; i += nwarp) {
        const C4 *v = V4 + (int64_t)i * K;
        C acc{0, 0};
#pragma unroll 4
        for (int q = lq; q < K; q += LQ) {
            const C4 vq = v[q];
            C t{0, 0};
            cfmac(t, C{vq.x, vq.y}, Gs[q * LB + lb]);
            cfmac(t, C{vq.z, vq.w}, Gs[(K + q) * LB + lb]);
            rfma(acc, lf.wq[q], t);
        }
#pragma unroll
        for (int off = 16; off >= LB; off >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
        }
        if (lq == 0 && lb < nb) {
            C y = yp[(int64_t)i * B + b0 + lb];
            y.x += acc.x;
            y.y += acc.y;
            yp[(int64_t)i * B + b0 + lb] = y;
        }
    }
}

// Many columns: one CTA per (leaf box, chunk of NB columns), samples in
// tiles of QT: the tile of G, of the weights and of every unknown's patterns
// go to shared memory by double-buffered asynchronous copies (the next
// tile's copies are in flight while this one is used); thread (row group,
// column) accumulates the rows i = group + k * groups of its column in
// registers.
template <class R, int NB, int MAXR>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 4 : 1) k_receive_tiled(const int32_t *__restrict__ box_ptr,
                                                       const typename Cx<R>::T4 *__restrict__ V4, DevLevel<R> lf,
                                                       typename Cx<R>::T *__restrict__ yp, int B, int Bs)
{
    using C = typename Cx<R>::T;
    using C4 = typename Cx<R>::T4;
    constexpr int QT = 16;
    constexpr int NG = 256 / NB;          // row groups
    constexpr int VP = QT + 1;            // padded row pitch of the pattern tile
    constexpr int GSZ = 2 * QT * NB, VSZ = NG * MAXR * VP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C4 *Vbuf = reinterpret_cast<C4 *>(smem_raw);                 // [2][VSZ]
    C *Gbuf = reinterpret_cast<C *>(Vbuf + 2 * VSZ);             // [2][GSZ]
    R *Wbuf = reinterpret_cast<R *>(Gbuf + 2 * GSZ);             // [2][QT]
    const int K = lf.K;
    // column chunk fastest in the grid: the CTAs that share a row's DRAM lines run together
    const int nch = (B + NB - 1) / NB, box = blockIdx.x / nch;
    const int b0 = (blockIdx.x - box * nch) * NB;
    const int bb = threadIdx.x % NB, grp = threadIdx.x / NB;
    const bool bok = b0 + bb < B;
    const int i0 = box_ptr[box], nrows = box_ptr[box + 1] - i0;
    const C *G = reinterpret_cast<const C *>(lf.G) + (int64_t)box * 2 * K * Bs + b0;
    const int ntile = (K + QT - 1) / QT;
    for (int r0 = 0; r0 < nrows; r0 += NG * MAXR) {
        const int nr = min(NG * MAXR, nrows - r0);
        auto stage = [&](int tile) {
            const int q0 = tile * QT, nq = min(QT, K - q0);
            C *Gs = Gbuf + (tile & 1) * GSZ;
            C4 *Vs = Vbuf + (tile & 1) * VSZ;
            R *Ws = Wbuf + (tile & 1) * QT;
            for (int e = threadIdx.x; e < GSZ; e += blockDim.x) {
                const int b = e % NB, q = (e / NB) % QT, cmp = e / (NB * QT);
                if (q < nq && b0 + b < B) cp_async(Gs + e, G + ((int64_t)cmp * K + q0 + q) * Bs + b);
                else Gs[e] = C{0, 0};
            }
            for (int e = threadIdx.x; e < nr * QT; e += blockDim.x) {
                const int r = e / QT, q = e % QT;
                C4 *d = Vs + r * VP + q;
                if (q < nq) {
                    const C4 *src = V4 + (int64_t)(i0 + r0 + r) * K + q0 + q;
#pragma unroll
                    for (int h = 0; h < (int)(sizeof(C4) / 16); ++h)
                        cp_async16(reinterpret_cast<char *>(d) + 16 * h, reinterpret_cast<const char *>(src) + 16 * h);
                } else {
                    *d = C4{0, 0, 0, 0};
                }
            }
            if (threadIdx.x < QT) Ws[threadIdx.x] = threadIdx.x < nq ? lf.wq[q0 + threadIdx.x] : R(0);
            cp_async_commit();
        };
        C acc[MAXR];
#pragma unroll
        for (int k = 0; k < MAXR; ++k) acc[k] = C{0, 0};
        stage(0);
        for (int tile = 0; tile < ntile; ++tile) {
            if (tile + 1 < ntile) {
                stage(tile + 1);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncthreads();
            const C *Gs = Gbuf + (tile & 1) * GSZ;
            const C4 *Vs = Vbuf + (tile & 1) * VSZ;
            const R *Ws = Wbuf + (tile & 1) * QT;
#pragma unroll 4
            for (int q = 0; q < QT; ++q) {
                const C g0 = Gs[q * NB + bb], g1 = Gs[(QT + q) * NB + bb];
                const R w = Ws[q];
#pragma unroll
                for (int k = 0; k < MAXR; ++k) {
                    const int r = grp + k * NG;
                    if (r >= nr) break;   // rows grow with k
                    const C4 v = Vs[r * VP + q];
                    C t{0, 0};
                    cfmac(t, C{v.x, v.y}, g0);
                    cfmac(t, C{v.z, v.w}, g1);
                    rfma(acc[k], w, t);
                }
            }
            __syncthreads();
        }
        if (bok) {
#pragma unroll
            for (int k = 0; k < MAXR; ++k) {
                const int r = grp + k * NG;
                if (r < nr) {
                    C *yv = yp + (int64_t)(i0 + r0 + r) * B + b0 + bb;
                    C y = *yv;
                    y.x += acc[k].x;
                    y.y += acc[k].y;
                    *yv = y;
                }
            }
        }
    }
}

// Radiation, many columns: thread (sample group, column) with QB samples in
// registers; x block of the box in shared memory.
template <class R, int NB, int QB>
__global__ void __launch_bounds__(256) k_radiate_tiled(const int32_t *__restrict__ box_ptr,
                                                       const typename Cx<R>::T4 *__restrict__ V4,
                                                       const R *__restrict__ xp, typename Cx<R>::T *__restrict__ S,
                                                       int K, int B, int Bs)
{
    using C = typename Cx<R>::T;
    using C4 = typename Cx<R>::T4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *xs = reinterpret_cast<R *>(smem_raw);   // [nj][NB]
    constexpr int NS = 256 / NB;
    // column chunk fastest in the grid: the CTAs that share a row's DRAM lines run together
    const int nch = (B + NB - 1) / NB, box = blockIdx.x / nch;
    const int b0 = (blockIdx.x - box * nch) * NB;
    const int bb = threadIdx.x % NB, slot = threadIdx.x / NB;
    const int j0 = box_ptr[box], nj = box_ptr[box + 1] - j0;
    for (int e = threadIdx.x; e < nj * NB; e += blockDim.x) {
        const int b = e % NB;
        xs[e] = b0 + b < B ? xp[(int64_t)(j0 + e / NB) * B + b0 + b] : R(0);
    }
    __syncthreads();
    const bool bok = b0 + bb < B;
    for (int qs = slot * QB; qs < K; qs += NS * QB) {
        C a0[QB], a1[QB];
#pragma unroll
        for (int k = 0; k < QB; ++k) a0[k] = a1[k] = C{0, 0};
        const C4 *vj = V4 + (int64_t)j0 * K + qs;
        for (int j = 0; j < nj; ++j) {
            const R xv = xs[j * NB + bb];
#pragma unroll
            for (int k = 0; k < QB; ++k) {
                if (qs + k < K) {
                    const C4 v = vj[(int64_t)j * K + k];
                    a0[k].x = fma(v.x, xv, a0[k].x);
                    a0[k].y = fma(v.y, xv, a0[k].y);
                    a1[k].x = fma(v.z, xv, a1[k].x);
                    a1[k].y = fma(v.w, xv, a1[k].y);
                }
            }
        }
        if (bok) {
#pragma unroll
            for (int k = 0; k < QB; ++k)
                if (qs + k < K) {
                    S[((int64_t)(box * 2 + 0) * K + qs + k) * Bs + b0 + bb] = a0[k];
                    S[((int64_t)(box * 2 + 1) * K + qs + k) * Bs + b0 + bb] = a1[k];
                }
        }
    }
}

// Radiation, all columns of a leaf box in one CTA (B a multiple of 4): the
// box's x block is staged once, the pattern tiles [rows x QT samples] by
// double-buffered asynchronous copies; thread (sample of the tile, group of
// 4 columns) accumulates both components of its 4 columns over the rows,
// from one broadcast pattern load and one 4-column x load per row.
template <class R>
__global__ void __launch_bounds__(256) k_radiate_wide(const int32_t *__restrict__ box_ptr,
                                                      const typename Cx<R>::T4 *__restrict__ V4,
                                                      const R *__restrict__ xp, typename Cx<R>::T *__restrict__ S,
                                                      int K, int B, int Bs, int max_rows)
{
    using C = typename Cx<R>::T;
    using C4 = typename Cx<R>::T4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ncg = B / 4, QT = blockDim.x / ncg;
    C4 *Vbuf = reinterpret_cast<C4 *>(smem_raw);                      // [2][max_rows][QT]
    R *xs = reinterpret_cast<R *>(Vbuf + (size_t)2 * max_rows * QT);  // [nj][B]
    const int box = blockIdx.x;
    const int j0 = box_ptr[box], nj = box_ptr[box + 1] - j0;
    const int t = threadIdx.x, cg = t % ncg, qi = t / ncg;
    constexpr int VEC = 16 / sizeof(R);
    for (int e = t; e < nj * (B / VEC); e += blockDim.x)
        cp_async16(xs + e * VEC, xp + (int64_t)j0 * B + e * VEC);
    const int ntile = (K + QT - 1) / QT;
    auto stage = [&](int tile) {
        const int q0 = tile * QT, nq = min(QT, K - q0);
        C4 *Vs = Vbuf + (size_t)(tile & 1) * max_rows * QT;
        for (int e = t; e < nj * QT; e += blockDim.x) {
            const int j = e / QT, q = e - j * QT;
            C4 *d = Vs + e;
            if (q < nq) {
                const C4 *src = V4 + (int64_t)(j0 + j) * K + q0 + q;
#pragma unroll
                for (int h = 0; h < (int)(sizeof(C4) / 16); ++h)
                    cp_async16(reinterpret_cast<char *>(d) + 16 * h, reinterpret_cast<const char *>(src) + 16 * h);
            } else {
                *d = C4{0, 0, 0, 0};
            }
        }
        cp_async_commit();
    };
    stage(0);   // the x block joins the first group
    for (int tile = 0; tile < ntile; ++tile) {
        if (tile + 1 < ntile) {
            stage(tile + 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const int q = tile * QT + qi;
        if (qi < QT && q < K) {
            const C4 *Vs = Vbuf + (size_t)(tile & 1) * max_rows * QT + qi;
            const R *xr = xs + cg * 4;
            C a0[4], a1[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) a0[k] = a1[k] = C{0, 0};
#pragma unroll 2
            for (int j = 0; j < nj; ++j) {
                const C4 v = Vs[j * QT];
                R xv[4];
                if constexpr (sizeof(R) == 4) {
                    const float4 x4 = *reinterpret_cast<const float4 *>(xr + j * B);
                    xv[0] = x4.x; xv[1] = x4.y; xv[2] = x4.z; xv[3] = x4.w;
                } else {
                    const double2 xa = *reinterpret_cast<const double2 *>(xr + j * B);
                    const double2 xb = *reinterpret_cast<const double2 *>(xr + j * B + 2);
                    xv[0] = xa.x; xv[1] = xa.y; xv[2] = xb.x; xv[3] = xb.y;
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    a0[k].x = fma(v.x, xv[k], a0[k].x);
                    a0[k].y = fma(v.y, xv[k], a0[k].y);
                    a1[k].x = fma(v.z, xv[k], a1[k].x);
                    a1[k].y = fma(v.w, xv[k], a1[k].y);
                }
            }
            C *s0 = S + ((int64_t)(box * 2 + 0) * K + q) * Bs + cg * 4;
            C *s1 = S + ((int64_t)(box * 2 + 1) * K + q) * Bs + cg * 4;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                s0[k] = a0[k];
                s1[k] = a1[k];
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------- launchers ---
template <class R, int BT>
cudaError_t launch_near_bt(const ProductArgs<R> &a, cudaStream_t s)
{
    using C = typename Cx<R>::T;
    dim3 grid(a.nr.nleaf * ((a.B + BT - 1) / BT));
    const size_t smem = (size_t)a.nr.max_cols * BT * sizeof(R);
    if (smem <= (size_t)kStageCap) {
        k_near<R, BT, true><<<grid, 256, smem, s>>>(a.nr, reinterpret_cast<const C *>(a.near_val), a.xp,
                                                    reinterpret_cast<C *>(a.yp), a.B);
    } else {
        k_near<R, BT, false><<<grid, 256, 0, s>>>(a.nr, reinterpret_cast<const C *>(a.near_val), a.xp,
                                                  reinterpret_cast<C *>(a.yp), a.B);
    }
    return cudaGetLastError();
}

template <class R, int BPT>
cudaError_t launch_near_wide(const ProductArgs<R> &a, cudaStream_t s)
{
    using C = typename Cx<R>::T;
    const size_t smem = (size_t)2 * 32 * (a.B * sizeof(R) + a.nr.max_rows * sizeof(C));
    k_near_wide<R, BPT><<<a.nr.nleaf, 256, smem, s>>>(a.nr, reinterpret_cast<const C *>(a.near_val), a.xp,
                                                      reinterpret_cast<C *>(a.yp), a.B);
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_near(const ProductArgs<R> &a, cudaStream_t s, int choice = 0)
{
    const bool wide_ok = a.B % 16 == 0 && a.nr.nleaf > 0 && a.B <= 512 &&
                         (size_t)2 * 32 * (a.B * sizeof(R) + a.nr.max_rows * sizeof(typename Cx<R>::T)) <= (size_t)kStageCap;
    if (choice == 1) return wide_ok ? launch_near_wide<R, 8>(a, s) : cudaErrorInvalidConfiguration;
    if (choice == 2) return wide_ok ? launch_near_wide<R, 16>(a, s) : cudaErrorInvalidConfiguration;
    if (choice == 3) return a.B >= 16 ? launch_near_bt<R, 16>(a, s) : cudaErrorInvalidConfiguration;
    // wide path: all columns per strip pass (B a multiple of 16 bytes of R and BPT)
    if (a.B >= 32 && wide_ok) {
        if (a.B <= 256) return launch_near_wide<R, 8>(a, s);   // 8 columns x rows per thread; row tiles of 256 / (B/8)
        return launch_near_wide<R, 16>(a, s);
    }
    if (a.B == 1) return launch_near_bt<R, 1>(a, s);
    if (a.B == 2) return launch_near_bt<R, 2>(a, s);
    if (a.B <= 4) return launch_near_bt<R, 4>(a, s);
    if (a.B <= 8 || sizeof(R) == 8) return launch_near_bt<R, 8>(a, s);
    return launch_near_bt<R, 16>(a, s);
}

template <class R, int NB, int QB>
cudaError_t launch_radiate_tiled(const ProductArgs<R> &a, int Bs, cudaStream_t s)
{
    using C = typename Cx<R>::T;
    using C4 = typename Cx<R>::T4;
    const DevLevel<R> &Lf = a.lv[a.leaf];
    const size_t smem = (size_t)a.nr.max_rows * NB * sizeof(R);
    if (smem > (size_t)kSmemCap) return cudaErrorInvalidConfiguration;
    dim3 grid(Lf.nbox * ((a.B + NB - 1) / NB));
    k_radiate_tiled<R, NB, QB><<<grid, 256, smem, s>>>(a.nr.box_ptr, reinterpret_cast<const C4 *>(a.V), a.xp,
                                                       reinterpret_cast<C *>(Lf.S), Lf.K, a.B, Bs);
    return cudaGetLastError();
}

// Bs: row stride of the outgoing field in columns (>= a.B)
template <class R>
cudaError_t launch_radiate(const ProductArgs<R> &a, int Bs, cudaStream_t s, int choice = 0)
{
    using C = typename Cx<R>::T;
    using C4 = typename Cx<R>::T4;
    const DevLevel<R> &Lf = a.lv[a.leaf];
    if (choice == 5) {   // four columns and two samples per thread, 64 columns per CTA (FP32)
        if constexpr (sizeof(R) == 4) return launch_radiate_quads(a, Bs, s);
        else return cudaErrorInvalidConfiguration;
    }
    if constexpr (sizeof(R) == 4) {
        if (choice == 0 && a.B >= 32) {   // built-in for wide batches
            const cudaError_t e = launch_radiate_quads(a, Bs, s);
            if (e != cudaErrorInvalidConfiguration) return e;
        }
    }
    if (choice >= 2 && choice <= 4) {
        const int nb = choice == 2 ? 32 : choice == 3 ? 16 : 8;
        if (a.B < nb || (size_t)a.nr.max_rows * nb * sizeof(R) > (size_t)kStageCap) return cudaErrorInvalidConfiguration;
        return nb == 32 ? launch_radiate_tiled<R, 32, 4>(a, Bs, s)
                        : nb == 16 ? launch_radiate_tiled<R, 16, 4>(a, Bs, s) : launch_radiate_tiled<R, 8, 4>(a, Bs, s);
    }
    if (choice == 1 || choice == 0) {
      if (a.B % 4 == 0 && a.B >= 16 && a.B <= 256 && (a.B * sizeof(R)) % 16 == 0) {
        const int QT = 256 / (a.B / 4);
        const size_t smem = (size_t)2 * a.nr.max_rows * QT * sizeof(C4) + (size_t)a.nr.max_rows * a.B * sizeof(R);
        if (smem <= (size_t)kStageCap) {
            k_radiate_wide<R><<<Lf.nbox, 256, smem, s>>>(a.nr.box_ptr, reinterpret_cast<const C4 *>(a.V), a.xp,
                                                         reinterpret_cast<C *>(Lf.S), Lf.K, a.B, Bs, a.nr.max_rows);
            return cudaGetLastError();
        }
      }
      if (choice == 1) return cudaErrorInvalidConfiguration;
    }
    if (a.B >= 32 && (size_t)a.nr.max_rows * 32 * sizeof(R) <= (size_t)kStageCap) return launch_radiate_tiled<R, 32, 4>(a, Bs, s);
    if (a.B >= 16 && (size_t)a.nr.max_rows * 16 * sizeof(R) <= (size_t)kStageCap) return launch_radiate_tiled<R, 16, 4>(a, Bs, s);
    if (a.B >= 8 && (size_t)a.nr.max_rows * 8 * sizeof(R) <= (size_t)kStageCap) return launch_radiate_tiled<R, 8, 4>(a, Bs, s);
    int Bt = std::min(a.B, 32);
    while (Bt > 1 && (size_t)a.nr.max_rows * Bt * sizeof(R) > (size_t)kStageCap) Bt /= 2;
    const size_t smem = (size_t)a.nr.max_rows * Bt * sizeof(R);
    dim3 grid(Lf.nbox * ((a.B + Bt - 1) / Bt));
    k_radiate<R><<<grid, 256, smem, s>>>(a.nr.box_ptr, reinterpret_cast<const C4 *>(a.V), a.xp,
                                         reinterpret_cast<C *>(Lf.S), Lf.K, a.B, Bt, Bs);
    return cudaGetLastError();
}

template <class R, int LB>
cudaError_t launch_receive_lb(const ProductArgs<R> &a, int Bs, cudaStream_t s)
{
    using C = typename Cx<R>::T;
    using C4 = typename Cx<R>::T4;
    const DevLevel<R> &Lf = a.lv[a.leaf];
    dim3 grid(Lf.nbox * ((a.B + LB - 1) / LB));
    const size_t smem = (size_t)2 * Lf.K * LB * sizeof(C);
    k_receive<R, LB><<<grid, 256, smem, s>>>(a.nr.box_ptr, reinterpret_cast<const C4 *>(a.V), Lf,
                                             reinterpret_cast<C *>(a.yp), a.B, Bs);
    return cudaGetLastError();
}

template <class R, int NB>
cudaError_t launch_receive_tiled(const ProductArgs<R> &a, int Bs, cudaStream_t s)
{
    using C = typename Cx<R>::T;
    using C4 = typename Cx<R>::T4;
    const DevLevel<R> &Lf = a.lv[a.leaf];
    dim3 grid(Lf.nbox * ((a.B + NB - 1) / NB));
    constexpr int NG = 256 / NB, MAXR = NB / 4, QT = 16;
    const size_t smem = 2 * ((size_t)NG * MAXR * (QT + 1) * sizeof(C4) + (size_t)2 * QT * NB * sizeof(C) + QT * sizeof(R));
    k_receive_tiled<R, NB, MAXR><<<grid, 256, smem, s>>>(a.nr.box_ptr, reinterpret_cast<const C4 *>(a.V), Lf,
                                                         reinterpret_cast<C *>(a.yp), a.B, Bs);
    return cudaGetLastError();
}

// Bs: row stride of the incoming field in columns (>= a.B)
template <class R>
cudaError_t launch_receive(const ProductArgs<R> &a, int Bs, cudaStream_t s, int choice = 0)
{
    using C = typename Cx<R>::T;
    if (choice >= 4 && choice <= 6) {   // two columns per thread, 64 / 32 / 16 columns per CTA (FP32)
        if constexpr (sizeof(R) == 4) return launch_receive_pairs(a, Bs, 64 >> (choice - 4), s);
        else return cudaErrorInvalidConfiguration;
    }
    if constexpr (sizeof(R) == 4)
        if (choice == 0 && a.B >= 32) return launch_receive_pairs(a, Bs, 32, s);   // built-in for wide batches
    if (choice == 1) return a.B >= 32 ? launch_receive_tiled<R, 32>(a, Bs, s) : cudaErrorInvalidConfiguration;
    if (choice == 2) return a.B >= 16 ? launch_receive_tiled<R, 16>(a, Bs, s) : cudaErrorInvalidConfiguration;
    if (choice == 3) return a.B >= 8 ? launch_receive_tiled<R, 8>(a, Bs, s) : cudaErrorInvalidConfiguration;
    if (a.B >= 32 && sizeof(R) == 4) return launch_receive_tiled<R, 32>(a, Bs, s);
    if (a.B >= 16) return launch_receive_tiled<R, 16>(a, Bs, s);
    if (a.B >= 8) return launch_receive_tiled<R, 8>(a, Bs, s);
    const int K = a.lv[a.leaf].K;
    int lb = 1;
    while (lb < a.B) lb *= 2;
    while (lb > 1 && (size_t)2 * K * lb * sizeof(C) > (size_t)kStageCap) lb /= 2;
    switch (lb) {
    case 1: return launch_receive_lb<R, 1>(a, Bs, s);
    case 2: return launch_receive_lb<R, 2>(a, Bs, s);
    default: return launch_receive_lb<R, 4>(a, Bs, s);
    }
}

// ---- upward: columns per CTA NB, parent theta rows split RS ways
template <class R, int NB, int PO, int RB = 1>
cudaError_t launch_up_nb(const DevLevel<R> &P, const DevLevel<R> &Ch, int B, int Bs, int acc, cudaStream_t s)
{
    using C = typename Cx<R>::T;
    auto smem_of = [&](int rs) {
        const int rows = up_band_rows(P.nth, rs, RB);
        return ((size_t)Ch.K + (size_t)rows * (Ch.nph + P.nph)) * NB * sizeof(C);
    };
    int RS = 1;
    while (RS < P.nth && smem_of(RS) > (size_t)(64 * 1024)) ++RS;
    if (smem_of(RS) > (size_t)kSmemCap) return cudaErrorInvalidConfiguration;
    const int64_t ctas = (int64_t)P.nbox * 2 * ((B + NB - 1) / NB);
    while (ctas * RS < 8 * 152 && 2 * RS <= P.nth / 2) RS *= 2;
    dim3 grid(P.nbox * ((B + NB - 1) / NB) * RS, 2);
    k_up<R, NB, PO, RB><<<grid, 256, smem_of(RS), s>>>(P, Ch, B, RS, Bs, acc);
    return cudaGetLastError();
}

// rb = 1: rows one at a time (the interpolation order's taps); rb = 2: rows
// in pairs (up2_taps, FP32)
template <class R, int NB>
cudaError_t launch_up_po(const DevLevel<R> &P, const DevLevel<R> &Ch, int B, int Bs, int acc, int order, cudaStream_t s,
                         int rb = 1)
{
    if (rb == 2) {
        if constexpr (sizeof(R) == 4) {
            if (!P.thu2 || !P.phu2) return cudaErrorInvalidConfiguration;
            switch (P.up2_taps) {
            case 12: return launch_up_nb<R, NB, 12, 2>(P, Ch, B, Bs, acc, s);
            case 16: return launch_up_nb<R, NB, 16, 2>(P, Ch, B, Bs, acc, s);
            default: return cudaErrorInvalidConfiguration;
            }
        } else {
            return cudaErrorInvalidConfiguration;
        }
    }
    switch (order) {
    case 4: return launch_up_nb<R, NB, 4>(P, Ch, B, Bs, acc, s);
    case 6: return launch_up_nb<R, NB, 6>(P, Ch, B, Bs, acc, s);
    case 8: return launch_up_nb<R, NB, 8>(P, Ch, B, Bs, acc, s);
    case 10: return launch_up_nb<R, NB, 10>(P, Ch, B, Bs, acc, s);
    case 12: return launch_up_nb<R, NB, 12>(P, Ch, B, Bs, acc, s);
    default: return cudaErrorInvalidValue;
    }
}

template <class R>
int column_chunk(int B, size_t per_col_bytes)
{
    int nb = 1;
    while (nb * 2 <= std::min(B, 16)) nb *= 2;
    while (nb > 1 && per_col_bytes * nb > (size_t)(64 * 1024)) nb /= 2;
    return nb;
}

// B columns of fields with row stride Bs; acc: add into the parent field
template <class R>
cudaError_t launch_up(const DevLevel<R> &P, const DevLevel<R> &Ch, int B, int Bs, int acc, cudaStream_t s,
                      int nb_choice = 0)
{
    using C = typename Cx<R>::T;
    if (nb_choice > 300) {   // 304, 308, 316 windowed FP32 kernel with 4 / 8 / 16 columns per CTA; 404, 408 the
                             // same with 4 / 8 columns and registers for one more CTA per SM; 704, 708, 716
                             // with the children that differ only in z sharing one phi step
        if constexpr (sizeof(R) == 4) return launch_up_win(P, Ch, B, Bs, acc, nb_choice - 300, s);
        else return cudaErrorInvalidConfiguration;
    }
    if constexpr (sizeof(R) == 4) {
        if (nb_choice == 0 && B >= 16) {   // built-in for wide batches: windowed with z pairs, 8 columns per CTA
            const cudaError_t e = launch_up_win(P, Ch, B, Bs, acc, 408, s);
            if (e != cudaErrorInvalidConfiguration) return e;
        }
    }
    const int order = P.up_order;
    int nb = column_chunk<R>(B, ((size_t)Ch.K + (size_t)P.nth * (Ch.nph + P.nph)) * sizeof(C));
    int rb = 1;
    if (nb_choice > 200) {   // 202 .. 216: rows in pairs, 2 .. 16 columns per CTA
        rb = 2;
        nb_choice -= 200;
    }
    if (nb_choice) {
        if (nb_choice > 16 || (nb_choice & (nb_choice - 1)) || nb_choice > std::max(1, B)) return cudaErrorInvalidConfiguration;
        nb = nb_choice;
    }
    switch (nb) {
    case 1: return launch_up_po<R, 1>(P, Ch, B, Bs, acc, order, s, rb);
    case 2: return launch_up_po<R, 2>(P, Ch, B, Bs, acc, order, s, rb);
    case 4: return launch_up_po<R, 4>(P, Ch, B, Bs, acc, order, s, rb);
    case 8: return launch_up_po<R, 8>(P, Ch, B, Bs, acc, order, s, rb);
    default: return launch_up_po<R, 16>(P, Ch, B, Bs, acc, order, s, rb);
    }
}

template <class R, int ES, int CB>
cudaError_t launch_translate_es(const DevLevel<R> &Lv, int B, int Bs, int acc, cudaStream_t s)
{
    using C = typename Cx<R>::T;
    const int outs = Lv.K * (B / CB);
    dim3 grid(Lv.nparent, (outs + 128 / ES - 1) / (128 / ES));
    // samples one CTA touches, at most (its outputs may straddle a sample)
    const int nq = std::min(Lv.K, (128 / ES - 1) / (B / CB) + 2);
    const size_t smem = (size_t)Lv.max_lty * nq * sizeof(C);
    if (Lv.lty && smem <= (size_t)48 * 1024)
        k_translate<R, ES, CB, true><<<grid, 128, smem, s>>>(Lv, B, Bs, acc);
    else
        k_translate<R, ES, CB, false><<<grid, 128, 0, s>>>(Lv, B, Bs, acc);
    return cudaGetLastError();
}

// Two columns per thread when B is even and there is enough parallelism;
// lanes per output grow until the level offers ~16 warps per SM.
template <class R>
cudaError_t launch_translate(const DevLevel<R> &Lv, int B, int Bs, int acc, cudaStream_t s, int choice = 0)
{
    if (choice >= 9 && choice <= 11) {   // four columns per thread, 64 / 32 / 16 columns per CTA
        if constexpr (sizeof(R) == 4) return launch_translate_quad(Lv, B, Bs, acc, 64 >> (choice - 9), s);
        else return cudaErrorInvalidConfiguration;
    }
    if constexpr (sizeof(R) == 4) {
        if (choice == 0 && B >= 16) {   // built-in for wide batches: four columns per thread
            const cudaError_t e = launch_translate_quad(Lv, B, Bs, acc, B >= 64 ? 64 : (B >= 32 ? 32 : 16), s);
            if (e != cudaErrorInvalidConfiguration) return e;
        }
    }
    if (choice == 7 || choice == 8) {
        using C = typename Cx<R>::T;
        if (!Lv.il_ptr) return cudaErrorInvalidConfiguration;
        constexpr int QC = 2;
        const size_t smem = (size_t)Lv.ntype * QC * sizeof(C);
        if (smem > (size_t)48 * 1024) return cudaErrorInvalidConfiguration;
        dim3 grid(Lv.nparent, (Lv.K + QC - 1) / QC);
        if (choice == 7) k_translate_cw<R, 2, QC><<<grid, 256, smem, s>>>(Lv, B, Bs, acc);
        else k_translate_cw<R, 1, QC><<<grid, 256, smem, s>>>(Lv, B, Bs, acc);
        return cudaGetLastError();
    }
    switch (choice) {
    case 1: return B % 2 == 0 ? launch_translate_es<R, 1, 2>(Lv, B, Bs, acc, s) : cudaErrorInvalidConfiguration;
    case 2: return launch_translate_es<R, 1, 1>(Lv, B, Bs, acc, s);
    case 3: return launch_translate_es<R, 2, 1>(Lv, B, Bs, acc, s);
    case 4: return launch_translate_es<R, 4, 1>(Lv, B, Bs, acc, s);
    case 5: return launch_translate_es<R, 8, 1>(Lv, B, Bs, acc, s);
    case 6: return launch_translate_es<R, 16, 1>(Lv, B, Bs, acc, s);
    default: break;
    }
    const bool pair = (B % 2 == 0) && (int64_t)Lv.nparent * ((Lv.K * (B / 2) + 31) / 32) >= 16 * 152;
    if (pair) return launch_translate_es<R, 1, 2>(Lv, B, Bs, acc, s);
    const int64_t warps1 = (int64_t)Lv.nparent * ((Lv.K * B + 31) / 32);
    int es = 1;
    while (es < 16 && warps1 * es < 16 * 152 && es * 2 <= std::max(1, Lv.max_grp / 4)) es *= 2;
    switch (es) {
    case 1: return launch_translate_es<R, 1, 1>(Lv, B, Bs, acc, s);
    case 2: return launch_translate_es<R, 2, 1>(Lv, B, Bs, acc, s);
    case 4: return launch_translate_es<R, 4, 1>(Lv, B, Bs, acc, s);
    case 8: return launch_translate_es<R, 8, 1>(Lv, B, Bs, acc, s);
    default: return launch_translate_es<R, 16, 1>(Lv, B, Bs, acc, s);
    }
}

// ---- downward: columns per CTA NB, anterpolation taps per row TM
template <class R, int NB, int TM, int RB>
cudaError_t launch_down_nb(const DevLevel<R> &P, const DevLevel<R> &Ch, int B, int Bs, size_t smem, cudaStream_t s)
{
    dim3 grid(Ch.nbox * ((B + NB - 1) / NB), 2);
    k_down<R, NB, TM, RB><<<grid, 256, smem, s>>>(P, Ch, B, Bs);
    return cudaGetLastError();
}

// RB = 1: rows one at a time (dn_taps); RB = 2: rows in pairs (dn2_taps, FP32)
template <class R, int NB>
cudaError_t launch_down_tm(const DevLevel<R> &P, const DevLevel<R> &Ch, int B, int Bs, size_t smem, cudaStream_t s,
                           int rb = 1)
{
    if (rb == 2) {
        if constexpr (sizeof(R) == 4) {
            if (!P.thd2 || !P.phd2) return cudaErrorInvalidConfiguration;
            switch (P.dn2_taps) {
            case 16: return launch_down_nb<R, NB, 16, 2>(P, Ch, B, Bs, smem, s);
            case 20: return launch_down_nb<R, NB, 20, 2>(P, Ch, B, Bs, smem, s);
            case 24: return launch_down_nb<R, NB, 24, 2>(P, Ch, B, Bs, smem, s);
            default: return cudaErrorInvalidConfiguration;
            }
        } else {
            return cudaErrorInvalidConfiguration;
        }
    }
    switch (P.dn_taps) {
    case 16: return launch_down_nb<R, NB, 16, 1>(P, Ch, B, Bs, smem, s);
    case 20: return launch_down_nb<R, NB, 20, 1>(P, Ch, B, Bs, smem, s);
    case 24: return launch_down_nb<R, NB, 24, 1>(P, Ch, B, Bs, smem, s);
    case 32: return launch_down_nb<R, NB, 32, 1>(P, Ch, B, Bs, smem, s);
    default: return cudaErrorInvalidValue;
    }
}

template <class R, int NB>
cudaError_t launch_down_pp(const DevLevel<R> &P, const DevLevel<R> &Ch, int B, int Bs, cudaStream_t s)
{
    using C = typename Cx<R>::T;
    const size_t per_col = ((size_t)2 * P.K + (size_t)P.nth + (size_t)P.nth * Ch.nph + (size_t)Ch.K) * sizeof(C);
    const size_t smem = per_col * NB;
    if (smem > (size_t)kSmemCap) return cudaErrorInvalidConfiguration;
    dim3 grid(P.nbox * ((B + NB - 1) / NB), 2);
    switch (P.dn_taps) {
    case 16: k_down_pp<R, NB, 16><<<grid, 256, smem, s>>>(P, Ch, B, Bs); break;
    case 20: k_down_pp<R, NB, 20><<<grid, 256, smem, s>>>(P, Ch, B, Bs); break;
    default: return cudaErrorInvalidConfiguration;
    }
    return cudaGetLastError();
}

// B columns of fields with row stride Bs, added into the child's incoming field
template <class R>
cudaError_t launch_down(const DevLevel<R> &P, const DevLevel<R> &Ch, int B, int Bs, cudaStream_t s, int nb_choice = 0)
{
    if (nb_choice > 300) {   // 304, 308, 316 windowed FP32 kernel with 4 / 8 / 16 columns per CTA; 404, 408 the
                             // same with 4 / 8 columns and registers for one more CTA per SM; 504, 508 one
                             // CTA per parent (its field loaded once for all children), 4 / 8 columns; 804, 808
                             // per pair of children that differ only in z (one phi step for both)
        if constexpr (sizeof(R) == 4) return launch_down_win(P, Ch, B, Bs, nb_choice - 300, s);
        else return cudaErrorInvalidConfiguration;
    }
    if constexpr (sizeof(R) == 4) {
        if (nb_choice == 0 && B >= 16) {   // built-in for wide batches: windowed with z pairs, 8 then 4 columns
            cudaError_t e = launch_down_win(P, Ch, B, Bs, 508, s);
            if (e != cudaErrorInvalidConfiguration) return e;
            e = launch_down_win(P, Ch, B, Bs, 504, s);
            if (e != cudaErrorInvalidConfiguration) return e;
        }
    }
    if (nb_choice == 104) return launch_down_pp<R, 4>(P, Ch, B, Bs, s);
    if (nb_choice == 108) return launch_down_pp<R, 8>(P, Ch, B, Bs, s);
    using C = typename Cx<R>::T;
    const size_t per_col = ((size_t)P.K + (size_t)P.nth + (size_t)P.nth * Ch.nph + (size_t)Ch.K) * sizeof(C);
    int nb = column_chunk<R>(B, per_col);
    int rb = 1;
    if (nb_choice > 200) {   // 204, 208, 216: rows in pairs, 4 / 8 / 16 columns per CTA
        rb = 2;
        nb_choice -= 200;
    }
    if (nb_choice) {
        if (nb_choice > 16 || (nb_choice & (nb_choice - 1)) || nb_choice > std::max(1, B)) return cudaErrorInvalidConfiguration;
        nb = nb_choice;
    }
    const size_t smem = per_col * nb;
    if (smem > (size_t)kSmemCap) return cudaErrorInvalidConfiguration;
    switch (nb) {
    case 1: return launch_down_tm<R, 1>(P, Ch, B, Bs, smem, s, rb);
    case 2: return launch_down_tm<R, 2>(P, Ch, B, Bs, smem, s, rb);
    case 4: return launch_down_tm<R, 4>(P, Ch, B, Bs, smem, s, rb);
    case 8: return launch_down_tm<R, 8>(P, Ch, B, Bs, smem, s, rb);
    default: return launch_down_tm<R, 16>(P, Ch, B, Bs, smem, s, rb);
    }
}

}  // namespace

// Raise the dynamic shared-memory limit of every kernel that stages data,
// once per process and device, before any launch or graph capture.
template <class R>
cudaError_t prime_kernels()
{
    cudaError_t e;
#define ALLOW(k) do { if ((e = allow_smem(k)) != cudaSuccess) return e; } while (0)
#define ALLOW_UP(NB) ALLOW((k_up<R, NB, 4>)); ALLOW((k_up<R, NB, 6>)); ALLOW((k_up<R, NB, 8>)); \
    ALLOW((k_up<R, NB, 10>)); ALLOW((k_up<R, NB, 12>)); ALLOW((k_down<R, NB, 16, 1>)); ALLOW((k_down<R, NB, 20, 1>)); \
    ALLOW((k_down<R, NB, 24, 1>)); ALLOW((k_down<R, NB, 32, 1>)); \
    if (sizeof(R) == 4) { ALLOW((k_down<R, NB, 16, 2>)); ALLOW((k_down<R, NB, 20, 2>)); ALLOW((k_down<R, NB, 24, 2>)); \
                          ALLOW((k_up<R, NB, 12, 2>)); ALLOW((k_up<R, NB, 16, 2>)); }
    ALLOW((k_near<R, 1, true>)); ALLOW((k_near<R, 2, true>)); ALLOW((k_near<R, 4, true>));
    ALLOW((k_near<R, 8, true>)); ALLOW((k_near<R, 16, true>));
    ALLOW((k_near_wide<R, 8>)); ALLOW((k_near_wide<R, 16>));
    ALLOW((k_down_pp<R, 4, 16>)); ALLOW((k_down_pp<R, 4, 20>)); ALLOW((k_down_pp<R, 8, 16>)); ALLOW((k_down_pp<R, 8, 20>));
    ALLOW(k_radiate<R>);
    ALLOW(k_radiate_wide<R>);
    ALLOW((k_radiate_tiled<R, 8, 4>)); ALLOW((k_radiate_tiled<R, 16, 4>)); ALLOW((k_radiate_tiled<R, 32, 4>));
    ALLOW((k_receive<R, 1>)); ALLOW((k_receive<R, 2>)); ALLOW((k_receive<R, 4>));
    ALLOW((k_receive_tiled<R, 8, 2>)); ALLOW((k_receive_tiled<R, 16, 4>)); ALLOW((k_receive_tiled<R, 32, 8>));
    ALLOW_UP(1); ALLOW_UP(2); ALLOW_UP(4); ALLOW_UP(8); ALLOW_UP(16);
#undef ALLOW_UP
#undef ALLOW
    if (sizeof(R) == 4) {
        if ((e = prime_win_kernels()) != cudaSuccess) return e;
        if ((e = prime_receive_pairs()) != cudaSuccess) return e;
        return prime_translate_quad();
    }
    return cudaSuccess;
}

template <class R>
cudaError_t launch_prepare(const ProductArgs<R> &a, const void *x_user, int x_complex, int Bu, int adjoint,
                           cudaStream_t s)
{
    k_prepare<R><<<blocks_for(a.n * a.B, 256), 256, 0, s>>>(static_cast<const R *>(x_user), x_complex, Bu, a.B,
                                                            a.perm, a.n, adjoint, a.xp);
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_finalize(const ProductArgs<R> &a, void *y_user, int x_complex, int Bu, int adjoint,
                            cudaStream_t s)
{
    using C = typename Cx<R>::T;
    k_finalize<R><<<blocks_for(a.n * Bu, 256), 256, 0, s>>>(reinterpret_cast<const C *>(a.yp), x_complex, Bu, a.B,
                                                            a.perm, a.n, adjoint, static_cast<C *>(y_user));
    return cudaGetLastError();
}

namespace {
inline cudaError_t tick(StageClock *clk, int stage, cudaStream_t s)
{
    if (!clk) return cudaSuccess;
    if (clk->n >= 96) return cudaErrorInvalidValue;
    clk->stage[clk->n] = stage;
    return cudaEventRecord(clk->ev[clk->n++], s);
}
}  // namespace

// One level of the up / down pass: the tensor-core kernels when the product
// asks for them and the level fits, else the CUDA-core kernels.
template <class R>
cudaError_t up_level(const ProductArgs<R> &a, int l, int B, cudaStream_t s, int choice)
{
    if constexpr (sizeof(R) == 4) {
        if (a.umma) {
            cudaError_t e = launch_up_umma(a.lv[l], a.lv[l + 1], B, B, 0, a.umma == 3, s);
            if (e != cudaErrorInvalidConfiguration) return e;
        }
    }
    return launch_up<R>(a.lv[l], a.lv[l + 1], B, B, 0, s, choice);
}

template <class R>
cudaError_t down_level(const ProductArgs<R> &a, int l, int B, cudaStream_t s, int choice)
{
    if constexpr (sizeof(R) == 4) {
        if (a.umma) {
            cudaError_t e = launch_down_umma(a.lv[l], a.lv[l + 1], B, B, a.umma == 3, s);
            if (e != cudaErrorInvalidConfiguration) return e;
        }
    }
    return launch_down<R>(a.lv[l], a.lv[l + 1], B, B, s, choice);
}

template <class R>
cudaError_t launch_core_streams(const ProductArgs<R> &a, const CoreStreams &cs, StageClock *clk)
{
    const int B = a.B, leaf = a.leaf, top = a.coarsest;
    const bool serial = clk != nullptr || cs.far == nullptr;
    cudaStream_t s0 = cs.main;
    cudaStream_t sf = serial ? s0 : cs.far;
    cudaStream_t st = serial ? s0 : cs.tr;
    cudaError_t e;
#define TRY(x) do { if ((e = (x)) != cudaSuccess) return e; } while (0)
    // events: 0 fork, 1 far done, 2 translations done, 3 + l outgoing field of level l ready
    if (!serial) {
        TRY(cudaEventRecord(cs.ev[0], s0));
        TRY(cudaStreamWaitEvent(sf, cs.ev[0], 0));
    }
    const Tuning &tu = a.tune;
    TRY(launch_near<R>(a, s0, tu.near));
    TRY(tick(clk, STAGE_NEAR, s0));
    if (leaf >= top) {
        TRY(launch_radiate<R>(a, B, sf, tu.radiate));
        TRY(tick(clk, STAGE_RADIATE, sf));
        if (!serial) {
            TRY(cudaEventRecord(cs.ev[3 + leaf], sf));
            TRY(cudaStreamWaitEvent(st, cs.ev[3 + leaf], 0));
        }
        TRY(launch_translate<R>(a.lv[leaf], B, B, 0, st, tu.tr[leaf]));
        TRY(tick(clk, STAGE_TRANSLATE + leaf, st));
        for (int l = leaf - 1; l >= top; --l) {
            TRY(up_level<R>(a, l, B, sf, tu.up_nb[l]));
            TRY(tick(clk, STAGE_UP + l, sf));
            if (l == top) {
                TRY(launch_translate<R>(a.lv[l], B, B, 0, sf, tu.tr[l]));
                TRY(tick(clk, STAGE_TRANSLATE + l, sf));
            } else {
                if (!serial) {
                    TRY(cudaEventRecord(cs.ev[3 + l], sf));
                    TRY(cudaStreamWaitEvent(st, cs.ev[3 + l], 0));
                }
                TRY(launch_translate<R>(a.lv[l], B, B, 0, st, tu.tr[l]));
                TRY(tick(clk, STAGE_TRANSLATE + l, st));
            }
        }
        if (!serial) {
            TRY(cudaEventRecord(cs.ev[2], st));
            TRY(cudaStreamWaitEvent(sf, cs.ev[2], 0));
        }
        for (int l = top; l < leaf; ++l) {
            TRY(down_level<R>(a, l, B, sf, tu.down_nb[l]));
            TRY(tick(clk, STAGE_DOWN + l, sf));
        }
        if (!serial) {
            TRY(cudaEventRecord(cs.ev[1], sf));
            TRY(cudaStreamWaitEvent(s0, cs.ev[1], 0));
        }
        TRY(launch_receive<R>(a, B, s0, tu.receive));
        TRY(tick(clk, STAGE_RECEIVE, s0));
    }
#undef TRY
    return cudaSuccess;
}

// The concurrent pass above; when a launch fails part way, the side streams
// are joined back into the main one (so that a stream capture in progress
// can end, and no stream is left forked) and the failure is returned.
template <class R>
cudaError_t launch_core(const ProductArgs<R> &a, const CoreStreams &cs, StageClock *clk)
{
    const cudaError_t e = launch_core_streams<R>(a, cs, clk);
    if (e != cudaSuccess && clk == nullptr && cs.far != nullptr) {
        const cudaStream_t side[2] = {cs.far, cs.tr};
        for (int i = 0; i < 2; ++i)
            if (side[i] && cudaEventRecord(cs.ev[62 + i], side[i]) == cudaSuccess)
                cudaStreamWaitEvent(cs.main, cs.ev[62 + i], 0);
    }
    return e;
}

// The k-derivative of the far pass, differentiated stage by stage with the
// samples, stencils and truncation fixed.  Each field row holds the value
// (columns [0, T)) and its k-tangent (columns [T, 2T)); every stage runs
// once over all 2T columns with its own table, then once more from the value
// half into the tangent half with the derivative of that table:
//   radiate    S = V x,                 S' = V' x
//   up         S_p' += sum_c shift'_pc Interp(S_c)
//   translate  G' += sum alpha' S
//   down       G_c' += Anterp(conj(shift'_pc) G_p)
//   receive    y += w conj(V) . G' + w conj(V' + (2/k) V) . G
// (the 2/k is the derivative of the far constant -k^2 eta / 4 pi over itself).
template <class R>
cudaError_t launch_core_dk(const ProductArgs<R> &a, cudaStream_t s, StageClock *clk)
{
    const int T = a.B, Bs = 2 * a.B, leaf = a.leaf;
    if (!a.near_dk || (leaf >= 2 && (!a.Vd || !a.Wd))) return cudaErrorInvalidValue;
    auto tangent = [&](R *f) { return f + 2 * (size_t)T; };   // T complex columns
    cudaError_t e;
#define TRY(x) do { if ((e = (x)) != cudaSuccess) return e; } while (0)
    {
        ProductArgs<R> an = a;
        an.near_val = a.near_dk;
        TRY(launch_near<R>(an, s));
        TRY(tick(clk, STAGE_NEAR, s));
    }
    if (leaf < 2) return cudaSuccess;
    {
        TRY(launch_radiate<R>(a, Bs, s));
        ProductArgs<R> ad = a;
        ad.V = a.Vd;
        ad.lv[leaf].S = tangent(a.lv[leaf].S);
        TRY(launch_radiate<R>(ad, Bs, s));
        TRY(tick(clk, STAGE_RADIATE, s));
    }
    auto translate = [&](int l) -> cudaError_t {
        cudaError_t e2 = launch_translate<R>(a.lv[l], Bs, Bs, 0, s);
        if (e2 != cudaSuccess) return e2;
        DevLevel<R> x = a.lv[l];
        x.alpha = a.lv[l].alpha_dk;
        x.G = tangent(a.lv[l].G);
        if ((e2 = launch_translate<R>(x, T, Bs, 1, s)) != cudaSuccess) return e2;
        return tick(clk, STAGE_TRANSLATE + l, s);
    };
    TRY(translate(leaf));
    for (int l = leaf - 1; l >= 2; --l) {
        TRY(launch_up<R>(a.lv[l], a.lv[l + 1], Bs, Bs, 0, s));
        DevLevel<R> px = a.lv[l];
        px.shift = a.lv[l].shift_dk;
        px.shift_xy = px.gam = nullptr;   // the split shift is the value's: no pair kernels here
        px.dgrp = nullptr;
        px.S = tangent(a.lv[l].S);
        TRY(launch_up<R>(px, a.lv[l + 1], T, Bs, 1, s));
        TRY(tick(clk, STAGE_UP + l, s));
        TRY(translate(l));
    }
    for (int l = 2; l < leaf; ++l) {
        TRY(launch_down<R>(a.lv[l], a.lv[l + 1], Bs, Bs, s));
        DevLevel<R> px = a.lv[l], cx = a.lv[l + 1];
        px.shift = a.lv[l].shift_dk;
        px.shift_xy = px.gam = nullptr;   // the split shift is the value's: no pair kernels here
        px.dgrp = nullptr;
        cx.G = tangent(a.lv[l + 1].G);
        TRY(launch_down<R>(px, cx, T, Bs, s));
        TRY(tick(clk, STAGE_DOWN + l, s));
    }
    {
        ProductArgs<R> at = a;
        at.lv[leaf].G = tangent(a.lv[leaf].G);
        TRY(launch_receive<R>(at, Bs, s));
        ProductArgs<R> aw = a;
        aw.V = a.Wd;
        TRY(launch_receive<R>(aw, Bs, s));
        TRY(tick(clk, STAGE_RECEIVE, s));
    }
#undef TRY
    return cudaSuccess;
}

template <class R>
cudaError_t launch_stage(const ProductArgs<R> &a, int stage, int choice, cudaStream_t s)
{
    const int B = a.B;
    if (stage == STAGE_NEAR) return launch_near<R>(a, s, choice);
    if (stage == STAGE_RADIATE) return launch_radiate<R>(a, B, s, choice);
    if (stage == STAGE_RECEIVE) return launch_receive<R>(a, B, s, choice);
    if (stage >= STAGE_UP && stage < STAGE_TRANSLATE) {
        const int l = stage - STAGE_UP;
        if (l < a.coarsest || l >= a.leaf) return cudaErrorInvalidValue;
        return launch_up<R>(a.lv[l], a.lv[l + 1], B, B, 0, s, choice);
    }
    if (stage >= STAGE_TRANSLATE && stage < STAGE_DOWN) {
        const int l = stage - STAGE_TRANSLATE;
        if (l < a.coarsest || l > a.leaf) return cudaErrorInvalidValue;
        return launch_translate<R>(a.lv[l], B, B, 0, s, choice);
    }
    if (stage >= STAGE_DOWN && stage < STAGE_RECEIVE) {
        const int l = stage - STAGE_DOWN;
        if (l < a.coarsest || l >= a.leaf) return cudaErrorInvalidValue;
        return launch_down<R>(a.lv[l], a.lv[l + 1], B, B, s, choice);
    }
    return cudaErrorInvalidValue;
}

template cudaError_t prime_kernels<float>();
template cudaError_t prime_kernels<double>();
template cudaError_t launch_prepare<float>(const ProductArgs<float> &, const void *, int, int, int, cudaStream_t);
template cudaError_t launch_prepare<double>(const ProductArgs<double> &, const void *, int, int, int, cudaStream_t);
template cudaError_t launch_finalize<float>(const ProductArgs<float> &, void *, int, int, int, cudaStream_t);
template cudaError_t launch_finalize<double>(const ProductArgs<double> &, void *, int, int, int, cudaStream_t);
template cudaError_t launch_core<float>(const ProductArgs<float> &, const CoreStreams &, StageClock *);
template cudaError_t launch_core<double>(const ProductArgs<double> &, const CoreStreams &, StageClock *);
template cudaError_t launch_core_dk<float>(const ProductArgs<float> &, cudaStream_t, StageClock *);
template cudaError_t launch_stage<float>(const ProductArgs<float> &, int, int, cudaStream_t);
template cudaError_t launch_stage<double>(const ProductArgs<double> &, int, int, cudaStream_t);
template cudaError_t launch_core_dk<double>(const ProductArgs<double> &, cudaStream_t, StageClock *);

}  // namespace mlfma
