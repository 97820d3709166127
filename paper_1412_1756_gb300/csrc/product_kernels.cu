// The multilevel fast multipole product y = Z x (Section III, Eq. (ZI)) as a
// chain of kernels, each templated on the real type R (float or double):
//
//   prepare      x (caller order) -> xp (leaf order, real columns)
//   near         y = Z_near x          first term of Eq. (ZI)
//   radiate      S_m = sum_j V_s,mj x_j         aggregation at the leaf level
//   up_theta/phi S_p = sum_c shift_pc Interp(S_c)  (Section III-C)
//   translate    G_m = sum_{m' in IL(m)} alpha_mm' S_m'  (Eq. (8))
//   down_phi/theta G_c += Anterp(conj(shift_pc) G_p)   (Section III-C)
//   receive      y_i += (-k^2 eta / 4 pi) sum_q w_q conj(V_s,mi) . G_m
//   finalize     y (leaf order, complex columns) -> caller order and type
//
// Fields are [box][component theta/phi][sample q][column b], b innermost,
// q theta-major.  All kernels are bandwidth- or latency-bound CUDA-core
// code: the per-sample products are diagonal (translation) or banded
// (local interpolation), not dense contractions.
#include "device.h"

#include <algorithm>

namespace mlfma {

namespace {

template <class R> struct Cx;
template <> struct Cx<float> { using T = float2; using T4 = float4; };
template <> struct Cx<double> { using T = double2; using T4 = double4_32a; };

template <class C> __device__ __forceinline__ C cm(C a, C b)
{
    return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
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

inline int blocks_for(int64_t total, int threads)
{
    int64_t b = (total + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 64));
}

#define GRID_STRIDE(idx, total) \
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (total); idx += (int64_t)gridDim.x * blockDim.x)

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
// One CTA per leaf box; the box's strip [rows x neighbour columns] is
// column-major, so threads (g, r) walking columns c = g, g + G, ... read
// consecutive addresses.  Partial sums over g are reduced in shared memory.
template <class R, int BT>
__global__ void __launch_bounds__(256) k_near(DevNear nr, const typename Cx<R>::T *__restrict__ val,
                                              const R *__restrict__ xp, typename Cx<R>::T *__restrict__ yp, int B)
{
    using C = typename Cx<R>::T;
    __shared__ C red[256];
    const int box = blockIdx.x;
    const int b0 = blockIdx.y * BT;
    const int r0 = nr.box_ptr[box];
    const int nrow = nr.box_ptr[box + 1] - r0;
    const int c0 = nr.col_ptr[box];
    const int ncol = nr.col_ptr[box + 1] - c0;
    const int64_t off = nr.strip_off[box];
    const int t = threadIdx.x;
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
            for (int c = g; c < ncol; c += G) {
                const C z = v[(int64_t)c * nrow];
                const R *xr = xp + (int64_t)nr.strip_col[c0 + c] * B + b0;
#pragma unroll
                for (int bb = 0; bb < BT; ++bb)
                    if (b0 + bb < B) rfma(acc[bb], xr[bb], z);
            }
        }
#pragma unroll
        for (int bb = 0; bb < BT; ++bb) {
            red[t] = active ? acc[bb] : C{0, 0};
            __syncthreads();
            if (t < RT && b0 + bb < B) {
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

// ------------------------------------------------------------ radiate ---
// S_m(q) = sum_{j in m} V_s,mj(q) x_j, both components from one 2-complex load.
template <class R>
__global__ void k_radiate(const int32_t *__restrict__ box_ptr, const typename Cx<R>::T4 *__restrict__ V4,
                          const R *__restrict__ xp, typename Cx<R>::T *__restrict__ S, int K, int B)
{
    using C = typename Cx<R>::T;
    using C4 = typename Cx<R>::T4;
    const int box = blockIdx.x;
    const int j0 = box_ptr[box], j1 = box_ptr[box + 1];
    for (int t = threadIdx.x; t < K * B; t += blockDim.x) {
        const int q = t / B, b = t % B;
        C a0{0, 0}, a1{0, 0};
        for (int j = j0; j < j1; ++j) {
            const C4 v = V4[(int64_t)j * K + q];
            const R xv = xp[(int64_t)j * B + b];
            a0.x = fma(v.x, xv, a0.x);
            a0.y = fma(v.y, xv, a0.y);
            a1.x = fma(v.z, xv, a1.x);
            a1.y = fma(v.w, xv, a1.y);
        }
        S[((int64_t)(box * 2 + 0) * K + q) * B + b] = a0;
        S[((int64_t)(box * 2 + 1) * K + q) * B + b] = a1;
    }
}

// ---------------------------------------------------------- translate ---
// Eq. (8) applied sample by sample: G_m(q) = sum_{m'} alpha_t(q) S_m'(q).
template <class R>
__global__ void k_translate(DevLevel<R> lv, int B)
{
    using C = typename Cx<R>::T;
    __shared__ int s_src[192], s_ty[192];
    const int m = blockIdx.x;
    const int e0 = lv.il_ptr[m], ne = lv.il_ptr[m + 1] - e0;
    for (int e = threadIdx.x; e < ne; e += blockDim.x) {
        s_src[e] = lv.il_src[e0 + e];
        s_ty[e] = lv.il_type[e0 + e];
    }
    __syncthreads();
    const int K = lv.K;
    const C *S = reinterpret_cast<const C *>(lv.S);
    const C *alpha = reinterpret_cast<const C *>(lv.alpha);
    C *G = reinterpret_cast<C *>(lv.G);
    for (int t = threadIdx.x; t < K * B; t += blockDim.x) {
        const int q = t / B, b = t % B;
        C a0{0, 0}, a1{0, 0};
        for (int e = 0; e < ne; ++e) {
            const C al = alpha[(int64_t)s_ty[e] * K + q];
            const int64_t base = ((int64_t)s_src[e] * 2 * K + q) * B + b;
            cfma(a0, al, S[base]);
            cfma(a1, al, S[base + (int64_t)K * B]);
        }
        G[((int64_t)m * 2 * K + q) * B + b] = a0;
        G[((int64_t)m * 2 * K + K + q) * B + b] = a1;
    }
}

// ----------------------------------------------------------- upward ---
// theta step for every child box c of level l+1: T[c][comp][tp][vc][b]
template <class R>
__global__ void k_up_theta(DevLevel<R> P, DevLevel<R> Ch, typename Cx<R>::T *__restrict__ T, int B)
{
    using C = typename Cx<R>::T;
    const C *S = reinterpret_cast<const C *>(Ch.S);
    const int nphc = Ch.nph, hc = nphc / 2, Kc = Ch.K, ntp = P.nth;
    const int64_t total = (int64_t)Ch.nbox * 2 * ntp * nphc * B;
    GRID_STRIDE(idx, total)
    {
        int64_t r = idx;
        const int b = (int)(r % B); r /= B;
        const int v = (int)(r % nphc); r /= nphc;
        const int tp = (int)(r % ntp); r /= ntp;
        const int64_t cc = r;   // c * 2 + comp
        const C *src = S + cc * Kc * B + b;
        C acc{0, 0};
        for (int e = P.thu_ptr[tp]; e < P.thu_ptr[tp + 1]; ++e) {
            const int vv = P.thu_refl[e] ? (v + hc) % nphc : v;
            rfma(acc, P.thu_c[e], src[((int64_t)P.thu_idx[e] * nphc + vv) * B]);
        }
        T[idx] = acc;
    }
}

// phi step, phase shift to the parent centre, sum over children
template <class R>
__global__ void k_up_phi(DevLevel<R> P, DevLevel<R> Ch, const typename Cx<R>::T *__restrict__ T, int B)
{
    using C = typename Cx<R>::T;
    C *S = reinterpret_cast<C *>(P.S);
    const C *shift = reinterpret_cast<const C *>(P.shift);
    const int nphp = P.nph, nphc = Ch.nph, ntp = P.nth, Kp = P.K;
    const int64_t total = (int64_t)P.nbox * 2 * Kp * B;
    GRID_STRIDE(idx, total)
    {
        int64_t r = idx;
        const int b = (int)(r % B); r /= B;
        const int q = (int)(r % Kp); r /= Kp;
        const int comp = (int)(r % 2);
        const int p = (int)(r / 2);
        const int tp = q / nphp, u = q % nphp;
        C acc{0, 0};
        for (int c = P.child_ptr[p]; c < P.child_ptr[p + 1]; ++c) {
            const C *src = T + (((int64_t)c * 2 + comp) * ntp + tp) * nphc * B + b;
            C s{0, 0};
            for (int e = P.phu_ptr[u]; e < P.phu_ptr[u + 1]; ++e) rfma(s, P.phu_c[e], src[(int64_t)P.phu_idx[e] * B]);
            cfma(acc, shift[(int64_t)Ch.octant[c] * Kp + q], s);
        }
        S[idx] = acc;
    }
}

// --------------------------------------------------------- downward ---
// phi step of the anterpolation (weighted transpose), after the conjugate
// phase shift from the parent centre to the child centre.
template <class R>
__global__ void k_down_phi(DevLevel<R> P, DevLevel<R> Ch, typename Cx<R>::T *__restrict__ U, int B)
{
    using C = typename Cx<R>::T;
    const C *G = reinterpret_cast<const C *>(P.G);
    const C *shift = reinterpret_cast<const C *>(P.shift);
    const int nphp = P.nph, nphc = Ch.nph, ntp = P.nth, Kp = P.K;
    const int64_t total = (int64_t)Ch.nbox * 2 * ntp * nphc * B;
    GRID_STRIDE(idx, total)
    {
        int64_t r = idx;
        const int b = (int)(r % B); r /= B;
        const int v = (int)(r % nphc); r /= nphc;
        const int tp = (int)(r % ntp); r /= ntp;
        const int comp = (int)(r % 2);
        const int c = (int)(r / 2);
        const int par = Ch.parent[c];
        const C *sh = shift + (int64_t)Ch.octant[c] * Kp + (int64_t)tp * nphp;
        const C *g = G + (((int64_t)par * 2 + comp) * Kp + (int64_t)tp * nphp) * B + b;
        C acc{0, 0};
        for (int e = P.phd_ptr[v]; e < P.phd_ptr[v + 1]; ++e) {
            const int u = P.phd_idx[e];
            C t{0, 0};
            cfmac(t, sh[u], g[(int64_t)u * B]);
            rfma(acc, P.phd_c[e], t);
        }
        U[idx] = acc;
    }
}

// theta step of the anterpolation, accumulated into the child's incoming field
template <class R>
__global__ void k_down_theta(DevLevel<R> P, DevLevel<R> Ch, const typename Cx<R>::T *__restrict__ U, int B)
{
    using C = typename Cx<R>::T;
    C *G = reinterpret_cast<C *>(Ch.G);
    const int nphc = Ch.nph, hc = nphc / 2, Kc = Ch.K, ntp = P.nth;
    const int64_t total = (int64_t)Ch.nbox * 2 * Kc * B;
    GRID_STRIDE(idx, total)
    {
        int64_t r = idx;
        const int b = (int)(r % B); r /= B;
        const int q = (int)(r % Kc); r /= Kc;
        const int64_t cc = r;   // c * 2 + comp
        const int j = q / nphc, v = q % nphc;
        const C *src = U + cc * ntp * nphc * B + b;
        C acc = G[idx];
        for (int e = P.thd_ptr[j]; e < P.thd_ptr[j + 1]; ++e) {
            const int vv = P.thd_refl[e] ? (v + hc) % nphc : v;
            rfma(acc, P.thd_c[e], src[((int64_t)P.thd_idx[e] * nphc + vv) * B]);
        }
        G[idx] = acc;
    }
}

// ------------------------------------------------------------ receive ---
// y_i += sum_q wq_q conj(V_s,mi(q)) . G_m(q); one warp per (unknown, group of
// LB columns); lanes split into LB column lanes x (32/LB) sample lanes,
// reduced with shuffles.
template <class R, int LB>
__global__ void k_receive(const int32_t *__restrict__ ubox, const typename Cx<R>::T4 *__restrict__ V4,
                          DevLevel<R> lf, typename Cx<R>::T *__restrict__ yp, int64_t n, int B)
{
    using C = typename Cx<R>::T;
    using C4 = typename Cx<R>::T4;
    constexpr int LQ = 32 / LB;
    const int nch = (B + LB - 1) / LB;
    const int lane = threadIdx.x & 31;
    const int lb = lane % LB, lq = lane / LB;
    const int K = lf.K;
    const C *G = reinterpret_cast<const C *>(lf.G);
    const int64_t nw = n * nch;
    for (int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; w < nw;
         w += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t i = w / nch;
        const int b = (int)(w % nch) * LB + lb;
        const bool ok = b < B;
        const int box = ubox[i];
        const C *g0 = G + (int64_t)box * 2 * K * B + (ok ? b : 0);
        C acc{0, 0};
        for (int q = lq; q < K; q += LQ) {
            const C4 v = V4[i * K + q];
            const R wq = lf.wq[q];
            C t{0, 0};
            cfmac(t, C{v.x, v.y}, g0[(int64_t)q * B]);
            cfmac(t, C{v.z, v.w}, g0[(int64_t)(K + q) * B]);
            rfma(acc, wq, t);
        }
#pragma unroll
        for (int off = 16; off >= LB; off >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
        }
        if (lq == 0 && ok) {
            C y = yp[i * B + b];
            y.x += acc.x;
            y.y += acc.y;
            yp[i * B + b] = y;
        }
    }
}

template <class R, int BT>
cudaError_t launch_near_bt(const ProductArgs<R> &a, cudaStream_t s)
{
    using C = typename Cx<R>::T;
    dim3 grid(a.nr.nleaf, (a.B + BT - 1) / BT);
    k_near<R, BT><<<grid, 256, 0, s>>>(a.nr, reinterpret_cast<const C *>(a.near_val), a.xp,
                                       reinterpret_cast<C *>(a.yp), a.B);
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_near(const ProductArgs<R> &a, cudaStream_t s)
{
    if (a.B == 1) return launch_near_bt<R, 1>(a, s);
    if (a.B == 2) return launch_near_bt<R, 2>(a, s);
    if (a.B <= 4) return launch_near_bt<R, 4>(a, s);
    return launch_near_bt<R, 8>(a, s);
}

template <class R, int LB>
cudaError_t launch_receive_lb(const ProductArgs<R> &a, cudaStream_t s)
{
    using C = typename Cx<R>::T;
    using C4 = typename Cx<R>::T4;
    const int nch = (a.B + LB - 1) / LB;
    const int64_t threads = a.n * nch * 32;
    k_receive<R, LB><<<blocks_for(threads, 256), 256, 0, s>>>(a.ubox, reinterpret_cast<const C4 *>(a.V),
                                                              a.lv[a.leaf], reinterpret_cast<C *>(a.yp), a.n, a.B);
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_receive(const ProductArgs<R> &a, cudaStream_t s)
{
    if (a.B <= 1) return launch_receive_lb<R, 1>(a, s);
    if (a.B <= 2) return launch_receive_lb<R, 2>(a, s);
    if (a.B <= 4) return launch_receive_lb<R, 4>(a, s);
    if (a.B <= 8) return launch_receive_lb<R, 8>(a, s);
    if (a.B <= 16) return launch_receive_lb<R, 16>(a, s);
    return launch_receive_lb<R, 32>(a, s);
}

}  // namespace

template <class R>
cudaError_t run_product(const ProductArgs<R> &a, const void *x_user, int x_complex, void *y_user, int Bu, int adjoint,
                        cudaStream_t s)
{
    using C = typename Cx<R>::T;
    using C4 = typename Cx<R>::T4;
    const int B = a.B;
    cudaError_t e;
    k_prepare<R><<<blocks_for(a.n * B, 256), 256, 0, s>>>(static_cast<const R *>(x_user), x_complex, Bu, B, a.perm,
                                                          a.n, adjoint, a.xp);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_near<R>(a, s)) != cudaSuccess) return e;
    const int leaf = a.leaf;
    if (leaf >= 2) {
        const DevLevel<R> &Lf = a.lv[leaf];
        k_radiate<R><<<Lf.nbox, 256, 0, s>>>(a.nr.box_ptr, reinterpret_cast<const C4 *>(a.V), a.xp,
                                             reinterpret_cast<C *>(Lf.S), Lf.K, B);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        C *T = reinterpret_cast<C *>(a.scratch);
        for (int l = leaf - 1; l >= 2; --l) {
            const DevLevel<R> &P = a.lv[l], &Ch = a.lv[l + 1];
            const int64_t nt = (int64_t)Ch.nbox * 2 * P.nth * Ch.nph * B;
            k_up_theta<R><<<blocks_for(nt, 256), 256, 0, s>>>(P, Ch, T, B);
            const int64_t np = (int64_t)P.nbox * 2 * P.K * B;
            k_up_phi<R><<<blocks_for(np, 256), 256, 0, s>>>(P, Ch, T, B);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        for (int l = 2; l <= leaf; ++l) {
            const DevLevel<R> &Lv = a.lv[l];
            k_translate<R><<<Lv.nbox, 256, 0, s>>>(Lv, B);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        for (int l = 2; l < leaf; ++l) {
            const DevLevel<R> &P = a.lv[l], &Ch = a.lv[l + 1];
            const int64_t nt = (int64_t)Ch.nbox * 2 * P.nth * Ch.nph * B;
            k_down_phi<R><<<blocks_for(nt, 256), 256, 0, s>>>(P, Ch, T, B);
            const int64_t nc = (int64_t)Ch.nbox * 2 * Ch.K * B;
            k_down_theta<R><<<blocks_for(nc, 256), 256, 0, s>>>(P, Ch, T, B);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        if ((e = launch_receive<R>(a, s)) != cudaSuccess) return e;
    }
    k_finalize<R><<<blocks_for(a.n * Bu, 256), 256, 0, s>>>(reinterpret_cast<const C *>(a.yp), x_complex, Bu, B,
                                                            a.perm, a.n, adjoint, static_cast<C *>(y_user));
    return cudaGetLastError();
}

template cudaError_t run_product<float>(const ProductArgs<float> &, const void *, int, void *, int, int, cudaStream_t);
template cudaError_t run_product<double>(const ProductArgs<double> &, const void *, int, void *, int, int,
                                         cudaStream_t);

}  // namespace mlfma
