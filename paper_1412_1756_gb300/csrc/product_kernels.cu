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

constexpr int kSmemCap = 96 * 1024;   // dynamic shared memory a kernel may ask for

inline int blocks_for(int64_t total, int threads)
{
    int64_t b = (total + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 64));
}

#define GRID_STRIDE(idx, total) \
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (total); idx += (int64_t)gridDim.x * blockDim.x)

template <class K>
cudaError_t allow_smem(K kernel)
{
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap);
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
    const int box = blockIdx.x;
    const int b0 = blockIdx.y * BT;
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

// ------------------------------------------------------------ radiate ---
// S_m(q) = sum_{j in m} V_s,mj(q) x_j for one leaf box and a chunk of
// columns; both components from one 2-complex load; x block in shared memory.
template <class R>
__global__ void __launch_bounds__(256) k_radiate(const int32_t *__restrict__ box_ptr,
                                                 const typename Cx<R>::T4 *__restrict__ V4,
                                                 const R *__restrict__ xp, typename Cx<R>::T *__restrict__ S,
                                                 int K, int B, int Bt)
{
    using C = typename Cx<R>::T;
    using C4 = typename Cx<R>::T4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *xs = reinterpret_cast<R *>(smem_raw);
    const int box = blockIdx.x;
    const int b0 = blockIdx.y * Bt;
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
        S[((int64_t)(box * 2 + 0) * K + q) * B + b0 + bb] = a0;
        S[((int64_t)(box * 2 + 1) * K + q) * B + b0 + bb] = a1;
    }
}

// ---------------------------------------------------------- translate ---
// Eq. (8) sample by sample, grouped by parent: the children of one parent
// draw on one candidate set (children of the parent's neighbours), so each
// source field value is loaded once and applied to every child whose
// interaction list holds it.  Each (sample q, column b) output is shared by
// ES consecutive lanes that split the source list and meet in a shuffle
// reduction (ES > 1 where outputs alone are too few to fill the GPU); all
// children's accumulators live in registers.
template <class R, int ES>
__global__ void __launch_bounds__(128) k_translate(DevLevel<R> lv, int B)
{
    using C = typename Cx<R>::T;
    __shared__ int s_src[216];
    __shared__ int16_t s_ty[216 * 8];
    const int P = blockIdx.x;
    const int e0 = lv.grp_ptr[P], ne = lv.grp_ptr[P + 1] - e0;
    const int m0 = lv.pchild_ptr[P], nc = lv.pchild_ptr[P + 1] - m0;
    for (int e = threadIdx.x; e < ne; e += blockDim.x) s_src[e] = lv.grp_src[e0 + e];
    for (int e = threadIdx.x; e < ne * 8; e += blockDim.x) s_ty[e] = lv.grp_ty[(int64_t)e0 * 8 + e];
    __syncthreads();
    const int K = lv.K;
    const int part = threadIdx.x % ES;
    const int t = blockIdx.y * (blockDim.x / ES) + threadIdx.x / ES;
    const bool valid = t < K * B;
    const int q = valid ? t / B : 0, b = valid ? t % B : 0;
    const C *S = reinterpret_cast<const C *>(lv.S);
    const C *alpha = reinterpret_cast<const C *>(lv.alpha) + q;
    C acc[8][2];
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c][0] = acc[c][1] = C{0, 0};
    const int64_t KB = (int64_t)K * B;
    const int64_t qb = (int64_t)q * B + b;
    if (valid) {
#pragma unroll 2
        for (int e = part; e < ne; e += ES) {
            const int64_t base = (int64_t)s_src[e] * 2 * KB + qb;
            const C s0 = S[base], s1 = S[base + KB];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int ty = s_ty[e * 8 + c];
                if (ty >= 0) {
                    const C al = alpha[(int64_t)ty * K];
                    cfma(acc[c][0], al, s0);
                    cfma(acc[c][1], al, s1);
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
                for (int k = 0; k < 2; ++k) {
                    acc[c][k].x += __shfl_xor_sync(0xffffffffu, acc[c][k].x, off);
                    acc[c][k].y += __shfl_xor_sync(0xffffffffu, acc[c][k].y, off);
                }
        }
    }
    if (!valid || part != 0) return;
    C *G = reinterpret_cast<C *>(lv.G);
#pragma unroll
    for (int c = 0; c < 8; ++c)
        if (c < nc) {
            const int64_t o = (int64_t)(m0 + c) * 2 * KB + qb;
            G[o] = acc[c][0];
            G[o + KB] = acc[c][1];
        }
}

// ----------------------------------------------------------- upward ---
// One CTA per (parent box, component, chunk of Bt columns): for each child,
// its field -> shared memory, theta interpolation -> shared memory, phi
// interpolation and phase shift accumulated in registers (MAXO outputs per
// thread).
template <class R, int MAXO>
__global__ void k_up(DevLevel<R> P, DevLevel<R> Ch, int B, int Bt, int RS)
{
    using C = typename Cx<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Kc = Ch.K, nphc = Ch.nph, hc = nphc / 2, ntp = P.nth, nphp = P.nph;
    const int p = blockIdx.x, comp = blockIdx.y;
    const int nbc = (B + Bt - 1) / Bt;
    const int bc = blockIdx.z % nbc, rs = blockIdx.z / nbc;
    const int b0 = bc * Bt, nb = min(Bt, B - b0);
    // this CTA's parent theta rows [t0, t1)
    const int rows = (ntp + RS - 1) / RS, t0 = rs * rows, t1 = min(ntp, t0 + rows);
    if (t0 >= t1) return;
    C *A = reinterpret_cast<C *>(smem_raw);          // [Kc][nb]
    C *T = A + (size_t)Kc * Bt;                       // [t1-t0][nphc][nb]
    const C *S = reinterpret_cast<const C *>(Ch.S);
    const C *shift = reinterpret_cast<const C *>(P.shift) + (int64_t)t0 * nphp;
    C acc[MAXO];
#pragma unroll
    for (int k = 0; k < MAXO; ++k) acc[k] = C{0, 0};
    const int Kp = (t1 - t0) * nphp;   // outputs of this CTA per column
    const int nout = Kp * nb;
    for (int c = P.child_ptr[p]; c < P.child_ptr[p + 1]; ++c) {
        const C *src = S + ((int64_t)c * 2 + comp) * Kc * B + b0;
        for (int e = threadIdx.x; e < Kc * nb; e += blockDim.x) A[e] = src[(int64_t)(e / nb) * B + e % nb];
        __syncthreads();
        for (int e = threadIdx.x; e < (t1 - t0) * nphc * nb; e += blockDim.x) {
            const int bb = e % nb, v = (e / nb) % nphc, tp = t0 + e / (nb * nphc);
            C s{0, 0};
            for (int f = P.thu_ptr[tp]; f < P.thu_ptr[tp + 1]; ++f) {
                const int vv = P.thu_refl[f] ? (v + hc) % nphc : v;
                rfma(s, P.thu_c[f], A[(P.thu_idx[f] * nphc + vv) * nb + bb]);
            }
            T[e] = s;
        }
        __syncthreads();
        const C *sh = shift + (int64_t)Ch.octant[c] * P.K;
#pragma unroll
        for (int k = 0; k < MAXO; ++k) {
            const int o = threadIdx.x + k * blockDim.x;
            if (o < nout) {
                const int q = o / nb, bb = o % nb;
                const int tp = q / nphp, u = q % nphp;   // tp relative to t0
                C s{0, 0};
                for (int f = P.phu_ptr[u]; f < P.phu_ptr[u + 1]; ++f)
                    rfma(s, P.phu_c[f], T[(tp * nphc + P.phu_idx[f]) * nb + bb]);
                cfma(acc[k], sh[q], s);
            }
        }
        __syncthreads();
    }
    C *dst = reinterpret_cast<C *>(P.S) + (((int64_t)p * 2 + comp) * P.K + (int64_t)t0 * nphp) * B + b0;
#pragma unroll
    for (int k = 0; k < MAXO; ++k) {
        const int o = threadIdx.x + k * blockDim.x;
        if (o < nout) dst[(int64_t)(o / nb) * B + o % nb] = acc[k];
    }
}

// --------------------------------------------------------- downward ---
// One CTA per (child box, component, chunk of Bt columns): parent field
// times the conjugate shift -> shared memory, phi anterpolation -> shared
// memory, theta anterpolation added into the child's incoming field.
template <class R>
__global__ void k_down(DevLevel<R> P, DevLevel<R> Ch, int B, int Bt)
{
    using C = typename Cx<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Kc = Ch.K, nphc = Ch.nph, hc = nphc / 2, ntp = P.nth, nphp = P.nph, Kp = P.K;
    const int c = blockIdx.x, comp = blockIdx.y;
    const int b0 = blockIdx.z * Bt, nb = min(Bt, B - b0);
    C *H = reinterpret_cast<C *>(smem_raw);          // [Kp][nb]
    C *U = H + (size_t)Kp * Bt;                       // [ntp][nphc][nb]
    const int par = Ch.parent[c];
    const C *g = reinterpret_cast<const C *>(P.G) + ((int64_t)par * 2 + comp) * Kp * B + b0;
    const C *sh = reinterpret_cast<const C *>(P.shift) + (int64_t)Ch.octant[c] * Kp;
    for (int e = threadIdx.x; e < Kp * nb; e += blockDim.x) {
        const int q = e / nb;
        C h{0, 0};
        cfmac(h, sh[q], g[(int64_t)q * B + e % nb]);
        H[e] = h;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < ntp * nphc * nb; e += blockDim.x) {
        const int bb = e % nb, v = (e / nb) % nphc, tp = e / (nb * nphc);
        C s{0, 0};
        for (int f = P.phd_ptr[v]; f < P.phd_ptr[v + 1]; ++f) rfma(s, P.phd_c[f], H[(tp * nphp + P.phd_idx[f]) * nb + bb]);
        U[e] = s;
    }
    __syncthreads();
    C *dst = reinterpret_cast<C *>(Ch.G) + ((int64_t)c * 2 + comp) * Kc * B + b0;
    for (int e = threadIdx.x; e < Kc * nb; e += blockDim.x) {
        const int bb = e % nb, q = e / nb;
        const int j = q / nphc, v = q % nphc;
        C s = dst[(int64_t)q * B + bb];
        for (int f = P.thd_ptr[j]; f < P.thd_ptr[j + 1]; ++f) {
            const int vv = P.thd_refl[f] ? (v + hc) % nphc : v;
            rfma(s, P.thd_c[f], U[(P.thd_idx[f] * nphc + vv) * nb + bb]);
        }
        dst[(int64_t)q * B + bb] = s;
    }
}

// ------------------------------------------------------------ receive ---
// y_i += sum_q wq_q conj(V_s,mi(q)) . G_m(q).  One CTA per (leaf box, chunk
// of LB columns) with the box's G block in shared memory; one warp per
// unknown at a time, lanes split into LB column lanes x 32/LB sample lanes,
// reduced with shuffles.
template <class R, int LB>
__global__ void __launch_bounds__(256) k_receive(const int32_t *__restrict__ box_ptr,
                                                 const typename Cx<R>::T4 *__restrict__ V4, DevLevel<R> lf,
                                                 typename Cx<R>::T *__restrict__ yp, int B)
{
    using C = typename Cx<R>::T;
    using C4 = typename Cx<R>::T4;
    constexpr int LQ = 32 / LB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *Gs = reinterpret_cast<C *>(smem_raw);   // [2][K][LB]
    const int K = lf.K;
    const int box = blockIdx.x;
    const int b0 = blockIdx.y * LB;
    const int nb = min(LB, B - b0);
    const C *G = reinterpret_cast<const C *>(lf.G) + (int64_t)box * 2 * K * B + b0;
    for (int e = threadIdx.x; e < 2 * K * LB; e += blockDim.x) {
        const int bb = e % LB;
        Gs[e] = bb < nb ? G[(int64_t)(e / LB) * B + bb] : C{0, 0};
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int lb = lane % LB, lq = lane / LB;
    const int i0 = box_ptr[box], i1 = box_ptr[box + 1];
    for (int i = i0 + warp; i < i1; i += nwarp) {
        const C4 *v = V4 + (int64_t)i * K;
        C acc{0, 0};
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

// ---------------------------------------------------------- launchers ---
template <class R, int BT>
cudaError_t launch_near_bt(const ProductArgs<R> &a, cudaStream_t s)
{
    using C = typename Cx<R>::T;
    dim3 grid(a.nr.nleaf, (a.B + BT - 1) / BT);
    const size_t smem = (size_t)a.nr.max_cols * BT * sizeof(R);
    if (smem <= (size_t)kSmemCap) {
        k_near<R, BT, true><<<grid, 256, smem, s>>>(a.nr, reinterpret_cast<const C *>(a.near_val), a.xp,
                                                    reinterpret_cast<C *>(a.yp), a.B);
    } else {
        k_near<R, BT, false><<<grid, 256, 0, s>>>(a.nr, reinterpret_cast<const C *>(a.near_val), a.xp,
                                                  reinterpret_cast<C *>(a.yp), a.B);
    }
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_near(const ProductArgs<R> &a, cudaStream_t s)
{
    if (a.B == 1) return launch_near_bt<R, 1>(a, s);
    if (a.B == 2) return launch_near_bt<R, 2>(a, s);
    if (a.B <= 4) return launch_near_bt<R, 4>(a, s);
    if (a.B <= 8 || sizeof(R) == 8) return launch_near_bt<R, 8>(a, s);
    return launch_near_bt<R, 16>(a, s);
}

template <class R>
cudaError_t launch_radiate(const ProductArgs<R> &a, cudaStream_t s)
{
    using C = typename Cx<R>::T;
    using C4 = typename Cx<R>::T4;
    const DevLevel<R> &Lf = a.lv[a.leaf];
    int Bt = std::min(a.B, 32);
    while (Bt > 1 && (size_t)a.nr.max_rows * Bt * sizeof(R) > (size_t)kSmemCap) Bt /= 2;
    const size_t smem = (size_t)a.nr.max_rows * Bt * sizeof(R);
    dim3 grid(Lf.nbox, (a.B + Bt - 1) / Bt);
    k_radiate<R><<<grid, 256, smem, s>>>(a.nr.box_ptr, reinterpret_cast<const C4 *>(a.V), a.xp,
                                         reinterpret_cast<C *>(Lf.S), Lf.K, a.B, Bt);
    return cudaGetLastError();
}

template <class R, int LB>
cudaError_t launch_receive_lb(const ProductArgs<R> &a, cudaStream_t s)
{
    using C = typename Cx<R>::T;
    using C4 = typename Cx<R>::T4;
    const DevLevel<R> &Lf = a.lv[a.leaf];
    dim3 grid(Lf.nbox, (a.B + LB - 1) / LB);
    const size_t smem = (size_t)2 * Lf.K * LB * sizeof(C);
    k_receive<R, LB><<<grid, 256, smem, s>>>(a.nr.box_ptr, reinterpret_cast<const C4 *>(a.V), Lf,
                                             reinterpret_cast<C *>(a.yp), a.B);
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_receive(const ProductArgs<R> &a, cudaStream_t s)
{
    using C = typename Cx<R>::T;
    const int K = a.lv[a.leaf].K;
    int lb = 1;
    while (lb < a.B && lb < 32) lb *= 2;
    while (lb > 1 && (size_t)2 * K * lb * sizeof(C) > (size_t)kSmemCap) lb /= 2;
    switch (lb) {
    case 1: return launch_receive_lb<R, 1>(a, s);
    case 2: return launch_receive_lb<R, 2>(a, s);
    case 4: return launch_receive_lb<R, 4>(a, s);
    case 8: return launch_receive_lb<R, 8>(a, s);
    case 16: return launch_receive_lb<R, 16>(a, s);
    default: return launch_receive_lb<R, 32>(a, s);
    }
}

template <class R, int MAXO>
cudaError_t launch_up_t(const DevLevel<R> &P, const DevLevel<R> &Ch, int B, int Bt, int RS, int nt, size_t smem,
                        cudaStream_t s)
{
    dim3 grid(P.nbox, 2, ((B + Bt - 1) / Bt) * RS);
    k_up<R, MAXO><<<grid, nt, smem, s>>>(P, Ch, B, Bt, RS);
    return cudaGetLastError();
}

// Column chunk Bt bounded by shared memory and by 16 register outputs per
// thread; the parent's theta rows split RS ways until there are enough CTAs.
template <class R>
cudaError_t launch_up(const DevLevel<R> &P, const DevLevel<R> &Ch, int B, cudaStream_t s)
{
    using C = typename Cx<R>::T;
    const int nt = P.K > 4096 ? 512 : 256;
    int Bt = std::min(B, 16), RS = 1;
    auto fits = [&](int bt, int rs) {
        const int rows = (P.nth + rs - 1) / rs;
        const size_t smem = ((size_t)Ch.K + (size_t)rows * Ch.nph) * bt * sizeof(C);
        return smem <= (size_t)kSmemCap && (rows * P.nph * bt + nt - 1) / nt <= 16;
    };
    while (Bt > 1 && !fits(Bt, RS)) --Bt;
    while (!fits(Bt, RS) && RS < P.nth) ++RS;
    if (!fits(Bt, RS)) return cudaErrorInvalidConfiguration;
    const int64_t ctas = (int64_t)P.nbox * 2 * ((B + Bt - 1) / Bt);
    while (ctas * RS < 4 * 152 && RS * 2 <= P.nth / 2) RS *= 2;
    const int rows = (P.nth + RS - 1) / RS;
    const size_t smem = ((size_t)Ch.K + (size_t)rows * Ch.nph) * Bt * sizeof(C);
    const int no = (rows * P.nph * Bt + nt - 1) / nt;
    if (no <= 4) return launch_up_t<R, 4>(P, Ch, B, Bt, RS, nt, smem, s);
    if (no <= 8) return launch_up_t<R, 8>(P, Ch, B, Bt, RS, nt, smem, s);
    return launch_up_t<R, 16>(P, Ch, B, Bt, RS, nt, smem, s);
}

template <class R, int ES>
cudaError_t launch_translate_es(const DevLevel<R> &Lv, int B, cudaStream_t s)
{
    dim3 grid(Lv.nparent, (Lv.K * B + 128 / ES - 1) / (128 / ES));
    k_translate<R, ES><<<grid, 128, 0, s>>>(Lv, B);
    return cudaGetLastError();
}

// Lanes per output grow until the level offers ~16 warps per SM.
template <class R>
cudaError_t launch_translate(const DevLevel<R> &Lv, int B, cudaStream_t s)
{
    const int64_t warps1 = (int64_t)Lv.nparent * ((Lv.K * B + 31) / 32);
    int es = 1;
    while (es < 16 && warps1 * es < 16 * 152 && es * 2 <= std::max(1, Lv.max_grp / 4)) es *= 2;
    switch (es) {
    case 1: return launch_translate_es<R, 1>(Lv, B, s);
    case 2: return launch_translate_es<R, 2>(Lv, B, s);
    case 4: return launch_translate_es<R, 4>(Lv, B, s);
    case 8: return launch_translate_es<R, 8>(Lv, B, s);
    default: return launch_translate_es<R, 16>(Lv, B, s);
    }
}

template <class R>
cudaError_t launch_down(const DevLevel<R> &P, const DevLevel<R> &Ch, int B, cudaStream_t s)
{
    using C = typename Cx<R>::T;
    const size_t per_col = ((size_t)P.K + (size_t)P.nth * Ch.nph) * sizeof(C);
    int Bt = std::min(B, 16);
    while (Bt > 1 && per_col * Bt > (size_t)kSmemCap) --Bt;
    if (per_col * Bt > (size_t)kSmemCap) return cudaErrorInvalidConfiguration;
    dim3 grid(Ch.nbox, 2, (B + Bt - 1) / Bt);
    k_down<R><<<grid, 256, per_col * Bt, s>>>(P, Ch, B, Bt);
    return cudaGetLastError();
}

}  // namespace

namespace {
inline cudaError_t tick(StageClock *clk, int stage, cudaStream_t s)
{
    if (!clk) return cudaSuccess;
    if (clk->n >= 96) return cudaErrorInvalidValue;
    clk->stage[clk->n] = stage;
    return cudaEventRecord(clk->ev[clk->n++], s);
}
}  // namespace

// Raise the dynamic shared-memory limit of every kernel that stages data,
// once per process and device, before any launch or graph capture.
template <class R>
cudaError_t prime_kernels()
{
    cudaError_t e;
#define ALLOW(k) do { if ((e = allow_smem(k)) != cudaSuccess) return e; } while (0)
    ALLOW((k_near<R, 1, true>)); ALLOW((k_near<R, 2, true>)); ALLOW((k_near<R, 4, true>));
    ALLOW((k_near<R, 8, true>)); ALLOW((k_near<R, 16, true>));
    ALLOW(k_radiate<R>);
    ALLOW((k_receive<R, 1>)); ALLOW((k_receive<R, 2>)); ALLOW((k_receive<R, 4>));
    ALLOW((k_receive<R, 8>)); ALLOW((k_receive<R, 16>)); ALLOW((k_receive<R, 32>));
    ALLOW((k_up<R, 4>)); ALLOW((k_up<R, 8>)); ALLOW((k_up<R, 16>));
    ALLOW(k_down<R>);
#undef ALLOW
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

template <class R>
cudaError_t launch_core(const ProductArgs<R> &a, const CoreStreams &cs, StageClock *clk)
{
    const int B = a.B, leaf = a.leaf;
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
    TRY(launch_near<R>(a, s0));
    TRY(tick(clk, STAGE_NEAR, s0));
    if (leaf >= 2) {
        TRY(launch_radiate<R>(a, sf));
        TRY(tick(clk, STAGE_RADIATE, sf));
        if (!serial) {
            TRY(cudaEventRecord(cs.ev[3 + leaf], sf));
            TRY(cudaStreamWaitEvent(st, cs.ev[3 + leaf], 0));
        }
        TRY(launch_translate<R>(a.lv[leaf], B, st));
        TRY(tick(clk, STAGE_TRANSLATE + leaf, st));
        for (int l = leaf - 1; l >= 2; --l) {
            TRY(launch_up<R>(a.lv[l], a.lv[l + 1], B, sf));
            TRY(tick(clk, STAGE_UP + l, sf));
            if (l == 2) {
                TRY(launch_translate<R>(a.lv[l], B, sf));
                TRY(tick(clk, STAGE_TRANSLATE + l, sf));
            } else {
                if (!serial) {
                    TRY(cudaEventRecord(cs.ev[3 + l], sf));
                    TRY(cudaStreamWaitEvent(st, cs.ev[3 + l], 0));
                }
                TRY(launch_translate<R>(a.lv[l], B, st));
                TRY(tick(clk, STAGE_TRANSLATE + l, st));
            }
        }
        if (!serial) {
            TRY(cudaEventRecord(cs.ev[2], st));
            TRY(cudaStreamWaitEvent(sf, cs.ev[2], 0));
        }
        for (int l = 2; l < leaf; ++l) {
            TRY(launch_down<R>(a.lv[l], a.lv[l + 1], B, sf));
            TRY(tick(clk, STAGE_DOWN + l, sf));
        }
        if (!serial) {
            TRY(cudaEventRecord(cs.ev[1], sf));
            TRY(cudaStreamWaitEvent(s0, cs.ev[1], 0));
        }
        TRY(launch_receive<R>(a, s0));
        TRY(tick(clk, STAGE_RECEIVE, s0));
    }
#undef TRY
    return cudaSuccess;
}

template cudaError_t prime_kernels<float>();
template cudaError_t prime_kernels<double>();
template cudaError_t launch_prepare<float>(const ProductArgs<float> &, const void *, int, int, int, cudaStream_t);
template cudaError_t launch_prepare<double>(const ProductArgs<double> &, const void *, int, int, int, cudaStream_t);
template cudaError_t launch_finalize<float>(const ProductArgs<float> &, void *, int, int, int, cudaStream_t);
template cudaError_t launch_finalize<double>(const ProductArgs<double> &, void *, int, int, int, cudaStream_t);
template cudaError_t launch_core<float>(const ProductArgs<float> &, const CoreStreams &, StageClock *);
template cudaError_t launch_core<double>(const ProductArgs<double> &, const CoreStreams &, StageClock *);

}  // namespace mlfma
