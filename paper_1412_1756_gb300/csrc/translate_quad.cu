// Translation of FP32 fields (Section III-A, Eq. (8): the incoming field of
// a box is the sum over its interaction list of the diagonal translation
// function times the source box's outgoing field, sample by sample), grouped
// by parent as the plan lists it: one entry names a source box and, for each
// child of the parent, the translation type it needs or none.
//
// A CTA takes one parent's children at QB samples and NB columns (128
// threads: thread = (sample, four adjacent columns)).  A thread loads a
// source value once per entry (both components of its four columns) and
// applies it to four children at a time from accumulators in registers, so
// each decoded coefficient feeds 32 FMAs; a parent with more than four
// children takes a second pass over its entries.  The coefficients of the
// parent's types at the CTA's samples are copied into shared memory first.
#include "device.h"

namespace mlfma {

namespace {

// acc (two complex columns) += a * s
__device__ __forceinline__ void cmac2(float4 &acc, float2 a, float4 s)
{
    acc.x = fmaf(a.x, s.x, fmaf(-a.y, s.y, acc.x));
    acc.y = fmaf(a.x, s.y, fmaf(a.y, s.x, acc.y));
    acc.z = fmaf(a.x, s.z, fmaf(-a.y, s.w, acc.z));
    acc.w = fmaf(a.x, s.w, fmaf(a.y, s.z, acc.w));
}

constexpr int kThreads = 128;
constexpr int kMaxEntries = 216;   // entries of one parent (the plan's bound)
constexpr int kCh = 4;             // children per pass
constexpr unsigned kNone = 0xffffu;   // (entry, child) slot without a translation

// Four columns of one field row: two 16-byte loads when all four exist and
// are aligned, else the existing ones (zero past the end).
__device__ __forceinline__ void ld_quad(const float2 *p, int cols, bool a16, float4 &lo, float4 &hi)
{
    if (cols == 4 && a16) {
        lo = reinterpret_cast<const float4 *>(p)[0];
        hi = reinterpret_cast<const float4 *>(p)[1];
        return;
    }
    float2 v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = k < cols ? p[k] : make_float2(0.f, 0.f);
    lo = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
    hi = make_float4(v[2].x, v[2].y, v[3].x, v[3].y);
}

__device__ __forceinline__ void st_quad(float2 *p, int cols, bool a16, float4 lo, float4 hi, int accumulate)
{
    if (cols == 4 && a16) {
        float4 *q = reinterpret_cast<float4 *>(p);
        if (accumulate) {
            const float4 a = q[0], b = q[1];
            lo.x += a.x; lo.y += a.y; lo.z += a.z; lo.w += a.w;
            hi.x += b.x; hi.y += b.y; hi.z += b.z; hi.w += b.w;
        }
        q[0] = lo;
        q[1] = hi;
        return;
    }
    const float2 v[4] = {make_float2(lo.x, lo.y), make_float2(lo.z, lo.w), make_float2(hi.x, hi.y), make_float2(hi.z, hi.w)};
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (k < cols) {
            float2 y = v[k];
            if (accumulate) {
                const float2 o = p[k];
                y.x += o.x;
                y.y += o.y;
            }
            p[k] = y;
        }
}

// FULL: every thread's four columns exist and are 16-byte aligned (B a
// multiple of NB, even row stride, aligned fields), so the loads and stores
// take the two-vector path without a run-time test.
template <int NB, bool FULL = false>
__global__ void __launch_bounds__(kThreads) k_translate_q4(DevLevel<float> lv, int B, int Bs, int accumulate)
{
    constexpr int NQD = NB / 4, QB = kThreads / NQD;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *s_al = reinterpret_cast<float2 *>(smem_raw);   // [local type][QB]
    __shared__ int64_t s_off[kMaxEntries];                  // offset of each entry's source field
    __shared__ __align__(16) uint16_t s_ty[kMaxEntries * 8];   // per (entry, child): its row of s_al, or kNone
    const int K = lv.K;
    const int64_t KB = (int64_t)K * Bs;
    const int P = blockIdx.x, q0 = blockIdx.y * QB, b0 = blockIdx.z * NB;
    const int nq = min(QB, K - q0), ncols = min(NB, B - b0);
    const int e0 = lv.grp_ptr[P], ne = lv.grp_ptr[P + 1] - e0;
    const int m0 = lv.pchild_ptr[P], nc = lv.pchild_ptr[P + 1] - m0;
    const int l0 = lv.lty_ptr[P], nl = lv.lty_ptr[P + 1] - l0;
    const bool a16 = FULL || ((Bs % 2) == 0 && ((reinterpret_cast<uintptr_t>(lv.S) | reinterpret_cast<uintptr_t>(lv.G)) & 15) == 0);
    const float2 *al = reinterpret_cast<const float2 *>(lv.alpha);
    for (int i = threadIdx.x; i < nl * QB; i += blockDim.x) {
        const int lt = i / QB, qq = i - lt * QB;
        s_al[i] = qq < nq ? al[(int64_t)lv.lty[l0 + lt] * K + q0 + qq] : make_float2(0.f, 0.f);
    }
    for (int e = threadIdx.x; e < ne; e += blockDim.x) s_off[e] = (int64_t)lv.grp_src[e0 + e] * 2 * KB;
    for (int e = threadIdx.x; e < ne * 8; e += blockDim.x) {
        const int t = lv.grp_lty[(int64_t)e0 * 8 + e];
        s_ty[e] = (uint16_t)(t < 0 ? kNone : (unsigned)(t * QB));   // t * QB < 2^16 (launcher's shared-memory bound)
    }
    __syncthreads();
    const int qq = threadIdx.x / NQD, qd = threadIdx.x - qq * NQD;
    const int cols = qq < nq ? (FULL ? 4 : max(0, min(4, ncols - 4 * qd))) : 0;
    if (!cols) return;
    const float2 *S = reinterpret_cast<const float2 *>(lv.S) + (int64_t)(q0 + qq) * Bs + b0 + 4 * qd;
    const float2 *alq = s_al + qq;
    for (int c0 = 0; c0 < nc; c0 += kCh) {
        float4 acc[kCh][2][2];
#pragma unroll
        for (int c = 0; c < kCh; ++c)
#pragma unroll
            for (int m = 0; m < 2; ++m) acc[c][m][0] = acc[c][m][1] = make_float4(0.f, 0.f, 0.f, 0.f);
        const int nch = min(kCh, nc - c0);
#pragma unroll 2
        for (int e = 0; e < ne; ++e) {
            const float2 *src = S + s_off[e];
            float4 s[2][2];
            if (FULL) {
                const float4 *p4 = reinterpret_cast<const float4 *>(src), *q4 = reinterpret_cast<const float4 *>(src + KB);
                s[0][0] = p4[0];
                s[0][1] = p4[1];
                s[1][0] = q4[0];
                s[1][1] = q4[1];
            } else {
                ld_quad(src, cols, a16, s[0][0], s[0][1]);
                ld_quad(src + KB, cols, a16, s[1][0], s[1][1]);
            }
            // the four children's coefficient rows (16-bit each) of this pass
            const uint2 tyv = *reinterpret_cast<const uint2 *>(&s_ty[e * 8 + c0]);
            const unsigned tw[2] = {tyv.x, tyv.y};
#pragma unroll
            for (int c = 0; c < kCh; ++c) {
                if (c >= nch) break;
                const unsigned off = (tw[c >> 1] >> (16 * (c & 1))) & 0xffffu;
                if (off != kNone) {
                    const float2 a = alq[off];
#pragma unroll
                    for (int m = 0; m < 2; ++m) {
                        cmac2(acc[c][m][0], a, s[m][0]);
                        cmac2(acc[c][m][1], a, s[m][1]);
                    }
                }
            }
        }
        float2 *G = reinterpret_cast<float2 *>(lv.G) + (int64_t)(q0 + qq) * Bs + b0 + 4 * qd;
#pragma unroll
        for (int c = 0; c < kCh; ++c) {
            if (c >= nch) break;
#pragma unroll
            for (int m = 0; m < 2; ++m)
                st_quad(G + ((int64_t)(m0 + c0 + c) * 2 + m) * KB, cols, a16, acc[c][m][0], acc[c][m][1], accumulate);
        }
    }
}

template <int NB>
cudaError_t translate_q4_nb(const DevLevel<float> &lv, int B, int Bs, int acc, cudaStream_t s)
{
    const bool full = B % NB == 0 && Bs % 2 == 0 &&
                      ((reinterpret_cast<uintptr_t>(lv.S) | reinterpret_cast<uintptr_t>(lv.G)) & 15) == 0;
    constexpr int QB = kThreads / (NB / 4);
    if (!lv.lty || !lv.grp_lty || lv.max_grp > kMaxEntries) return cudaErrorInvalidConfiguration;
    const size_t smem = (size_t)lv.max_lty * QB * sizeof(float2);
    if (smem > (size_t)(96 * 1024)) return cudaErrorInvalidConfiguration;
    dim3 grid(lv.nparent, (lv.K + QB - 1) / QB, (B + NB - 1) / NB);
    if (full) k_translate_q4<NB, true><<<grid, kThreads, smem, s>>>(lv, B, Bs, acc);
    else k_translate_q4<NB, false><<<grid, kThreads, smem, s>>>(lv, B, Bs, acc);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_translate_quad(const DevLevel<float> &lv, int B, int Bs, int acc, int nb, cudaStream_t s)
{
    if (B < 1) return cudaErrorInvalidConfiguration;
    switch (nb) {
    case 16: return translate_q4_nb<16>(lv, B, Bs, acc, s);
    case 32: return translate_q4_nb<32>(lv, B, Bs, acc, s);
    case 64: return translate_q4_nb<64>(lv, B, Bs, acc, s);
    default: return cudaErrorInvalidConfiguration;
    }
}

cudaError_t prime_translate_quad()
{
    cudaError_t e;
#define ALLOW(k) do { if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024)) != cudaSuccess) return e; } while (0)
    ALLOW((k_translate_q4<16, false>)); ALLOW((k_translate_q4<32, false>)); ALLOW((k_translate_q4<64, false>));
    ALLOW((k_translate_q4<16, true>)); ALLOW((k_translate_q4<32, true>)); ALLOW((k_translate_q4<64, true>));
#undef ALLOW
    return cudaSuccess;
}

}  // namespace mlfma
