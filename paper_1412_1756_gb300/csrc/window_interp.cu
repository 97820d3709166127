// Interpolation (up pass) and anterpolation (down pass) of FP32 fields on
// CUDA cores with the stencil rows in groups of four on windows of
// consecutive source positions (Section III-C: local Lagrange interpolation
// between the levels' sampling grids, the theta component continued past
// the poles by F(-theta, phi) = -F(theta, phi + pi); the anterpolation is
// the weighted transpose).
//
// A warp takes one group of four output rows and a block of lines (the
// lane grid is column pairs x lines): at each window position the group's
// four coefficients are one broadcast shared-memory load, the source value
// of a lane (two adjacent field columns, 16 bytes) is one shared-memory load
// at a fixed offset from the window start, and it feeds the four rows - 16
// FMAs per 16-byte load.  Phi windows wrap around the periodic grid (two
// address segments); theta windows run over the reflected rows near a pole
// (reversed order, the column at phi + pi), the direct rows and the other
// pole's reflected rows (three segments).  No table is read from global
// memory inside the stencil loops: the coefficients and window starts are
// copied into shared memory once per CTA.
#include "device.h"

#include <algorithm>

namespace mlfma {

namespace {

constexpr int kG = 4;   // stencil rows per group

__device__ __forceinline__ void cp8(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// acc[r] += c[r] * a: a holds two complex columns (re0, im0, re1, im1).
__device__ __forceinline__ void fma_group(float4 (&acc)[kG], const float4 c, const float4 a)
{
    const float cc[kG] = {c.x, c.y, c.z, c.w};
#pragma unroll
    for (int r = 0; r < kG; ++r) {
        acc[r].x = fmaf(cc[r], a.x, acc[r].x);
        acc[r].y = fmaf(cc[r], a.y, acc[r].y);
        acc[r].z = fmaf(cc[r], a.z, acc[r].z);
        acc[r].w = fmaf(cc[r], a.w, acc[r].w);
    }
}

// Periodic window: positions s .. s + tw - 1 (mod n) of a line whose element
// e is line[e * ES]; tw <= n, 0 <= s < n.
template <int ES>
__device__ __forceinline__ void win_periodic(float4 (&acc)[kG], const float4 *cf, int tw, int s, int n,
                                             const float4 *line)
{
    const int seg = min(tw, n - s);
    const float4 *p = line + s * ES;
#pragma unroll 4
    for (int f = 0; f < seg; ++f) fma_group(acc, cf[f], p[f * ES]);
    const float4 *cf2 = cf + seg;
#pragma unroll 4
    for (int f = 0; f < tw - seg; ++f) fma_group(acc, cf2[f], line[f * ES]);
}

// Theta window: positions e = s + f (f < tw) over n rows of stride rs
// (float4); e < 0: row -e-1 from `ref` (the column at phi + pi), 0 <= e < n:
// row e from `dir`, e >= n: row 2n-e-1 from `ref`; -n <= s, s + tw <= 2n.
__device__ __forceinline__ void win_theta(float4 (&acc)[kG], const float4 *cf, int tw, int s, int n,
                                          const float4 *dir, const float4 *ref, int rs)
{
    const int fa = min(tw, max(0, -s));       // north reflection: f in [0, fa)
    const int fb = min(tw, max(0, n - s));    // direct: f in [fa, fb); south: [fb, tw)
    if (fa > 0) {
        const float4 *p = ref + (-s - 1) * rs;   // row -s-1-f
        for (int f = 0; f < fa; ++f) fma_group(acc, cf[f], p[-f * rs]);
    }
    if (fb > fa) {
        const float4 *p = dir + (s + fa) * rs;
        const float4 *c = cf + fa;
#pragma unroll 4
        for (int f = 0; f < fb - fa; ++f) fma_group(acc, c[f], p[f * rs]);
    }
    if (tw > fb) {
        const float4 *p = ref + (2 * n - s - fb - 1) * rs;   // row 2n-s-1-f for f >= fb
        const float4 *c = cf + fb;
        for (int f = 0; f < tw - fb; ++f) fma_group(acc, c[f], p[-f * rs]);
    }
}

// Shared-memory bytes of the coefficient and window-start copies.
__host__ __device__ inline size_t win_table_bytes(const WinDev &a, const WinDev &b)
{
    return ((size_t)a.groups * a.tw + (size_t)b.groups * b.tw) * sizeof(float4) +
           (size_t)(a.groups + b.groups) * sizeof(int32_t);
}

// Copies one table (coefficients cp.async, starts plain) into shared memory.
__device__ __forceinline__ void stage_table(const WinDev &w, float4 *cf, int *st)
{
    for (int i = threadIdx.x; i < w.groups * w.tw; i += blockDim.x) cp16(cf + i, w.coef + i);
    for (int i = threadIdx.x; i < w.groups; i += blockDim.x) st[i] = w.start[i];
}

// Walks q = q0, q0 + dq, ... over a row-major grid of n columns as
// (row t, column u), without a division per step.
struct Walk {
    int t, u, dt, du, n;
    __device__ Walk(int q0, int dq, int n_) : n(n_)
    {
        t = q0 / n;
        u = q0 - t * n;
        dt = dq / n;
        du = dq - dt * n;
    }
    __device__ void next()
    {
        t += dt;
        u += du;
        if (u >= n) {
            u -= n;
            ++t;
        }
    }
};

// Work items (group g, block of lines) of a stencil step, taken by warp w,
// w + nw, ... in g-major order without a division per step.
struct Items {
    int g, blk, dg, db, G;
    __device__ Items(int w, int nw, int groups) : G(groups)
    {
        g = w % G;
        blk = w / G;
        dg = nw % G;
        db = nw / G;
    }
    __device__ void next()
    {
        g += dg;
        blk += db;
        if (g >= G) {
            g -= G;
            ++blk;
        }
    }
};

// Column pairs of a chunk: the pair a thread copies (its first column 2 pc)
// and how many of its two columns exist (2, 1 or 0).
__device__ __forceinline__ int pair_cols(int pc, int nb) { return 2 * pc + 1 < nb ? 2 : (2 * pc < nb ? 1 : 0); }

// Asynchronous copy of one column pair of a field row into shared memory
// (16 bytes when both columns exist and the row stride keeps them 16-byte
// aligned; missing columns are zero).
__device__ __forceinline__ void cp_pair(float4 *d, const float2 *src, int cols, bool a16)
{
    if (cols == 2 && a16) {
        cp16(d, src);
    } else if (cols >= 1) {
        cp8(d, src);
        if (cols == 2) cp8(reinterpret_cast<float2 *>(d) + 1, src + 1);
        else reinterpret_cast<float2 *>(d)[1] = make_float2(0.f, 0.f);
    } else {
        *d = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}
__device__ __forceinline__ float4 ld_pair(const float2 *src, int cols, bool a16)
{
    if (cols == 2 && a16) return *reinterpret_cast<const float4 *>(src);
    const float2 a = cols >= 1 ? src[0] : make_float2(0.f, 0.f), b = cols == 2 ? src[1] : make_float2(0.f, 0.f);
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void st_pair(float2 *dst, float4 v, int cols, bool a16)
{
    if (cols == 2 && a16) {
        *reinterpret_cast<float4 *>(dst) = v;
    } else {
        if (cols >= 1) dst[0] = make_float2(v.x, v.y);
        if (cols == 2) dst[1] = make_float2(v.z, v.w);
    }
}

// ---------------------------------------------------------- downward ---
// One CTA per (child box, component, chunk of NB columns), 256 threads.
// The parent's incoming field is copied (cp.async, column pairs) into H
// (rows padded by one element, so the lines a warp reads fall in different
// banks) and multiplied by the conjugate shift in place; phi anterpolation
// H -> U (lines = parent theta rows; U rows padded likewise for the warp's
// stores); theta anterpolation U -> W (lines = child phi index; W over H);
// the child's own incoming field, requested before the theta step, plus W
// is stored back.
constexpr int kPF = 4;   // column pairs of the child's own field prefetched per thread

// The phi anterpolation step of one child (shared by the per-child and the
// per-parent kernels): H (shifted parent, rows padded to nphp + 1) -> U (rows
// padded to nphc + 1).
template <int NB>
__device__ __forceinline__ void down_phi(const float4 *H4, float4 *U4, const float4 *cph, const int *sph,
                                         const WinDev &wp, int ntp, int nphp, int nphc)
{
    constexpr int NCP = NB / 2, RL = 32 / NCP, ES = NB / 2;
    const int hp = nphp + 1, up = nphc + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int cpi = lane % NCP, rl = lane / NCP;
    // U(tp, v) = sum_f c H(tp, (s + f) mod nphp); lines tp, groups of child phi v
    const int blocks = (ntp + RL - 1) / RL;
    for (Items it(warp, nw, wp.groups); it.blk < blocks; it.next()) {
        const int g = it.g, tp = it.blk * RL + rl;
        const int tl = min(tp, ntp - 1);
        float4 acc[kG];
#pragma unroll
        for (int r = 0; r < kG; ++r) acc[r] = make_float4(0.f, 0.f, 0.f, 0.f);
        win_periodic<ES>(acc, cph + g * wp.tw, wp.tw, sph[g], nphp, H4 + (size_t)tl * hp * NCP + cpi);
        if (tp < ntp) {
#pragma unroll
            for (int r = 0; r < kG; ++r) {
                const int v = g * kG + r;
                if (v < nphc) U4[((size_t)tp * up + v) * NCP + cpi] = acc[r];
            }
        }
    }
}

// The theta anterpolation step: U -> W (unpadded [Kc][NCP]).
template <int NB>
__device__ __forceinline__ void down_theta(const float4 *U4, float4 *W4, const float4 *cth, const int *sth,
                                           const WinDev &wt, int ntp, int nthc, int nphc)
{
    constexpr int NCP = NB / 2, RL = 32 / NCP;
    const int up = nphc + 1, hc = nphc / 2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int cpi = lane % NCP, rl = lane / NCP;
    // theta: W(j, v) = sum_f c U(row of s + f, v or v + pi); lines v, groups of child theta j
    const int blocks = (nphc + RL - 1) / RL;
    for (Items it(warp, nw, wt.groups); it.blk < blocks; it.next()) {
        const int g = it.g, v = it.blk * RL + rl;
        const int vl = min(v, nphc - 1), vr = vl + hc < nphc ? vl + hc : vl + hc - nphc;
        float4 acc[kG];
#pragma unroll
        for (int r = 0; r < kG; ++r) acc[r] = make_float4(0.f, 0.f, 0.f, 0.f);
        win_theta(acc, cth + g * wt.tw, wt.tw, sth[g], ntp, U4 + vl * NCP + cpi, U4 + vr * NCP + cpi, up * NCP);
        if (v < nphc) {
#pragma unroll
            for (int r = 0; r < kG; ++r) {
                const int j = g * kG + r;
                if (j < nthc) W4[((size_t)j * nphc + v) * NCP + cpi] = acc[r];
            }
        }
    }
}

// dst (the child's incoming field, this thread's column pair) += W; the
// first PF pairs were prefetched into xin.
template <int NB, int PF>
__device__ __forceinline__ void down_add(float2 *dst, const float4 *W4, const float4 (&xin)[PF], int Kc, int Bs,
                                         int cols, bool a16)
{
    constexpr int NCP = NB / 2;
    const int pc = threadIdx.x % NCP, pslot = threadIdx.x / NCP, npslot = blockDim.x / NCP;
    if (!cols) return;
#pragma unroll
    for (int k = 0; k < PF; ++k) {
        const int q = pslot + k * npslot;
        if (q < Kc) {
            const float4 w = W4[q * NCP + pc], x = xin[k];
            st_pair(dst + (int64_t)q * Bs, make_float4(x.x + w.x, x.y + w.y, x.z + w.z, x.w + w.w), cols, a16);
        }
    }
#pragma unroll 4
    for (int q = pslot + PF * npslot; q < Kc; q += npslot) {
        const float4 w = W4[q * NCP + pc], x = ld_pair(dst + (int64_t)q * Bs, cols, a16);
        st_pair(dst + (int64_t)q * Bs, make_float4(x.x + w.x, x.y + w.y, x.z + w.z, x.w + w.w), cols, a16);
    }
}

template <int NB, int PF>
__device__ __forceinline__ void down_prefetch(float4 (&xin)[PF], const float2 *dst, int Kc, int Bs, int cols, bool a16)
{
    constexpr int NCP = NB / 2;
    const int pslot = threadIdx.x / NCP, npslot = blockDim.x / NCP;
#pragma unroll
    for (int k = 0; k < PF; ++k) {
        const int q = pslot + k * npslot;
        xin[k] = q < Kc ? ld_pair(dst + (int64_t)q * Bs, cols, a16) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// PAIR: a CTA takes a down-pass group of the parent level (two siblings that
// differ only in z, or one child).  The conjugate shift factors as
// conj(shift_xy) * conj(gam(theta)); the parent is shifted by the pair's
// common conj(shift_xy) and anterpolated in phi once, and each child's theta
// step runs on U with its rows scaled by that child's conj(gam).
template <int NB, int MINB, bool PAIR = false>
__global__ void __launch_bounds__(256, MINB) k_down_win(DevLevel<float> P, DevLevel<float> Ch, int B, int Bs)
{
    constexpr int NCP = NB / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Kc = Ch.K, nthc = Ch.nth, nphc = Ch.nph, ntp = P.nth, nphp = P.nph, Kp = P.K;
    const WinDev wp = P.wd_ph, wt = P.wd_th;
    // column chunk fastest in the grid: the CTAs that share a field row's DRAM lines run together
    const int nbc = (B + NB - 1) / NB, item = blockIdx.x / nbc, comp = blockIdx.y, b0 = (blockIdx.x - item * nbc) * NB;
    int ca = item, cb = -1;
    if (PAIR) {
        const int2 gp = P.dgrp[item];
        ca = gp.x;
        cb = gp.y;
    }
    const int nb = min(NB, B - b0);
    const int hp = nphp + 1, up = nphc + 1;
    float4 *H4 = reinterpret_cast<float4 *>(smem_raw);   // [ntp][hp][NCP]; then W [Kc][NCP]
    float4 *U4 = H4 + (size_t)ntp * hp * NCP;             // [ntp][up][NCP]
    float4 *cph = U4 + (size_t)ntp * up * NCP;
    float4 *cth = cph + wp.groups * wp.tw;
    int *sph = reinterpret_cast<int *>(cth + wt.groups * wt.tw);
    int *sth = sph + wp.groups;
    const int pc = threadIdx.x % NCP, pslot = threadIdx.x / NCP, npslot = blockDim.x / NCP;
    const int cols = pair_cols(pc, nb);
    const bool a16 = (Bs % 2) == 0 && ((reinterpret_cast<uintptr_t>(P.G) | reinterpret_cast<uintptr_t>(Ch.G)) & 15) == 0;
    const bool pair = PAIR && cb >= 0;
    {
        const int par = Ch.parent[ca];
        const float2 *g = reinterpret_cast<const float2 *>(P.G) + ((int64_t)par * 2 + comp) * Kp * Bs + b0 + 2 * pc;
        Walk w(pslot, npslot, nphp);
        for (int q = pslot; q < Kp; q += npslot, w.next()) cp_pair(H4 + (w.t * hp + w.u) * NCP + pc, g + (int64_t)q * Bs, cols, a16);
        stage_table(wp, cph, sph);
        stage_table(wt, cth, sth);
        cp_commit();
        const float2 *sh = reinterpret_cast<const float2 *>(pair ? P.shift_xy : P.shift) + (int64_t)Ch.octant[ca] * Kp;
        cp_wait<0>();
        Walk w2(pslot, npslot, nphp);
#pragma unroll 4
        for (int q = pslot; q < Kp; q += npslot, w2.next()) {   // the pairs this thread copied
            float4 *d = H4 + (w2.t * hp + w2.u) * NCP + pc;
            const float2 z = sh[q];
            const float4 h = *d;
            *d = make_float4(fmaf(z.x, h.x, z.y * h.y), fmaf(z.x, h.y, -z.y * h.x), fmaf(z.x, h.z, z.y * h.w),
                             fmaf(z.x, h.w, -z.y * h.z));
        }
    }
    __syncthreads();
    down_phi<NB>(H4, U4, cph, sph, wp, ntp, nphp, nphc);
    __syncthreads();
    constexpr int PF = MINB >= 4 ? 1 : kPF;   // fewer prefetch registers for the tighter budget
    const int nch = pair ? 2 : 1;
    for (int k = 0; k < nch; ++k) {
        const int c = k ? cb : ca;
        float2 *dst = reinterpret_cast<float2 *>(Ch.G) + ((int64_t)c * 2 + comp) * Kc * Bs + b0 + 2 * pc;
        if (pair) {
            // U rows times conj(gam_a) for the first child, then times gam_a conj(gam_b) for the second
            const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
            const float2 *ga = reinterpret_cast<const float2 *>(P.gam) + (int64_t)Ch.octant[ca] * ntp;
            const float2 *gb = reinterpret_cast<const float2 *>(P.gam) + (int64_t)Ch.octant[cb] * ntp;
            for (int t = warp; t < ntp; t += nw) {
                const float2 a = ga[t];
                float2 f = make_float2(a.x, -a.y);
                if (k) {
                    const float2 b = gb[t];   // a * conj(b)
                    f = make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
                }
                float4 *row = U4 + (size_t)t * up * NCP;
                for (int i = lane; i < nphc * NCP; i += 32) {
                    const float4 u = row[i];
                    row[i] = make_float4(f.x * u.x - f.y * u.y, f.x * u.y + f.y * u.x, f.x * u.z - f.y * u.w,
                                         f.x * u.w + f.y * u.z);
                }
            }
            __syncthreads();
        }
        float4 xin[PF];
        down_prefetch<NB, PF>(xin, dst, Kc, Bs, cols, a16);
        down_theta<NB>(U4, H4, cth, sth, wt, ntp, nthc, nphc);
        __syncthreads();
        down_add<NB, PF>(dst, H4, xin, Kc, Bs, cols, a16);
        if (k + 1 < nch) __syncthreads();   // W (over H) and U are read before the second child rewrites them
    }
}

// One CTA per (parent box, component, chunk of NB columns), 256 threads:
// the parent's incoming field is copied into shared memory once (R, rows
// padded) and each child in turn takes it through the shift (R -> H), the
// two anterpolation steps and the addition into its own field, so siblings
// do not fetch the parent again.
template <int NB, int MINB>
__global__ void __launch_bounds__(256, MINB) k_down_win_pp(DevLevel<float> P, DevLevel<float> Ch, int B, int Bs)
{
    constexpr int NCP = NB / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Kc = Ch.K, nthc = Ch.nth, nphc = Ch.nph, ntp = P.nth, nphp = P.nph, Kp = P.K;
    const WinDev wp = P.wd_ph, wt = P.wd_th;
    const int nbc = (B + NB - 1) / NB, p = blockIdx.x / nbc, comp = blockIdx.y, b0 = (blockIdx.x - p * nbc) * NB;
    const int nb = min(NB, B - b0);
    const int hp = nphp + 1, up = nphc + 1;
    float4 *R4 = reinterpret_cast<float4 *>(smem_raw);   // [ntp][hp][NCP] the parent as loaded
    float4 *H4 = R4 + (size_t)ntp * hp * NCP;             // [ntp][hp][NCP] shifted; then W [Kc][NCP]
    float4 *U4 = H4 + (size_t)ntp * hp * NCP;             // [ntp][up][NCP]
    float4 *cph = U4 + (size_t)ntp * up * NCP;
    float4 *cth = cph + wp.groups * wp.tw;
    int *sph = reinterpret_cast<int *>(cth + wt.groups * wt.tw);
    int *sth = sph + wp.groups;
    const int pc = threadIdx.x % NCP, pslot = threadIdx.x / NCP, npslot = blockDim.x / NCP;
    const int cols = pair_cols(pc, nb);
    const bool a16 = (Bs % 2) == 0 && ((reinterpret_cast<uintptr_t>(P.G) | reinterpret_cast<uintptr_t>(Ch.G)) & 15) == 0;
    {
        const float2 *g = reinterpret_cast<const float2 *>(P.G) + ((int64_t)p * 2 + comp) * Kp * Bs + b0 + 2 * pc;
        Walk w(pslot, npslot, nphp);
        for (int q = pslot; q < Kp; q += npslot, w.next()) cp_pair(R4 + (w.t * hp + w.u) * NCP + pc, g + (int64_t)q * Bs, cols, a16);
        stage_table(wp, cph, sph);
        stage_table(wt, cth, sth);
        cp_commit();
    }
    constexpr int PF = MINB >= 4 ? 1 : kPF;
    const int c0 = P.child_ptr[p], c1 = P.child_ptr[p + 1];
    for (int c = c0; c < c1; ++c) {
        float2 *dst = reinterpret_cast<float2 *>(Ch.G) + ((int64_t)c * 2 + comp) * Kc * Bs + b0 + 2 * pc;
        const float2 *sh = reinterpret_cast<const float2 *>(P.shift) + (int64_t)Ch.octant[c] * Kp;
        cp_wait<0>();
        if (c == c0) __syncthreads();   // the tables (copied by other threads) are in
        Walk w(pslot, npslot, nphp);
#pragma unroll 4
        for (int q = pslot; q < Kp; q += npslot, w.next()) {   // the pairs this thread copied
            const int i = (w.t * hp + w.u) * NCP + pc;
            const float2 z = sh[q];
            const float4 h = R4[i];
            H4[i] = make_float4(fmaf(z.x, h.x, z.y * h.y), fmaf(z.x, h.y, -z.y * h.x), fmaf(z.x, h.z, z.y * h.w),
                                fmaf(z.x, h.w, -z.y * h.z));
        }
        __syncthreads();
        down_phi<NB>(H4, U4, cph, sph, wp, ntp, nphp, nphc);
        __syncthreads();
        float4 xin[PF];
        down_prefetch<NB, PF>(xin, dst, Kc, Bs, cols, a16);
        down_theta<NB>(U4, H4, cth, sth, wt, ntp, nthc, nphc);
        __syncthreads();
        down_add<NB, PF>(dst, H4, xin, Kc, Bs, cols, a16);
        __syncthreads();   // W (over H) is read before the next child's shift writes H
    }
}

// ------------------------------------------------------------ upward ---
// One CTA per (parent box, component, chunk of NB columns, band of parent
// theta groups), 256 threads.  Per child: its outgoing field A and its
// octant's shift Z (band rows) arrive by cp.async - the next child's A is
// requested as soon as the theta step has read the current one, its Z as
// soon as the phi step has - then theta interpolation A -> T (lines = child
// phi index; T rows padded by one element), phi interpolation of T with the
// shift accumulated into O (lines = band rows; O and Z rows padded); one
// store of the parent's band at the end.
// PAIR: two children that differ only in their z octant bit (adjacent in the
// child order) share one phi step.  The shift factors as shift_xy(theta, phi)
// * gam(theta), and gam commutes with the phi interpolation, so the first
// child's T is scaled by its gam, the second's is scaled and added, and the
// phi step of the sum is accumulated with the pair's common shift_xy.
template <int NB, int MINB, bool PAIR = false>
__global__ void __launch_bounds__(256, MINB) k_up_win(DevLevel<float> P, DevLevel<float> Ch, int B, int RS, int Bs,
                                                      int accumulate)
{
    constexpr int NCP = NB / 2, RL = 32 / NCP, ES = NB / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Kc = Ch.K, nthc = Ch.nth, nphc = Ch.nph, hc = nphc / 2, ntp = P.nth, nphp = P.nph, Kp = P.K;
    const WinDev wt = P.wu_th, wp = P.wu_ph;
    // column chunk fastest in the grid, then the band, then the parent
    const int nbc = (B + NB - 1) / NB, comp = blockIdx.y;
    const int p = blockIdx.x / (nbc * RS), rem = blockIdx.x - p * (nbc * RS), band = rem / nbc, b0 = (rem - band * nbc) * NB;
    const int gpb = (wt.groups + RS - 1) / RS, g0 = band * gpb, g1 = min(wt.groups, g0 + gpb);
    if (g0 >= g1) return;
    const int t0 = g0 * kG, t1 = min(ntp, g1 * kG), nr = t1 - t0;
    const int nb = min(NB, B - b0);
    const int tpit = nphc + 1, opit = nphp + 1;
    float4 *A4 = reinterpret_cast<float4 *>(smem_raw);   // [Kc][NCP]
    float4 *T4 = A4 + (size_t)Kc * NCP;                  // [nr][tpit][NCP]
    float4 *O4 = T4 + (size_t)nr * tpit * NCP;           // [nr][opit][NCP]
    float2 *Z = reinterpret_cast<float2 *>(O4 + (size_t)nr * opit * NCP);   // [nr][opit]
    float4 *cth = reinterpret_cast<float4 *>((reinterpret_cast<uintptr_t>(Z + (size_t)nr * opit) + 15) & ~uintptr_t(15));
    float4 *cph = cth + (g1 - g0) * wt.tw;
    int *sth = reinterpret_cast<int *>(cph + wp.groups * wp.tw);
    int *sph = sth + (g1 - g0);
    const int pc = threadIdx.x % NCP, pslot = threadIdx.x / NCP, npslot = blockDim.x / NCP;
    const int cols = pair_cols(pc, nb);
    const bool a16 = (Bs % 2) == 0 && ((reinterpret_cast<uintptr_t>(P.S) | reinterpret_cast<uintptr_t>(Ch.S)) & 15) == 0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const float2 *S = reinterpret_cast<const float2 *>(Ch.S);
    const float2 *shift = reinterpret_cast<const float2 *>(P.shift) + (int64_t)t0 * nphp;
    const float2 *shift_xy = reinterpret_cast<const float2 *>(P.shift_xy) + (int64_t)t0 * nphp;
    const float2 *gam = reinterpret_cast<const float2 *>(P.gam) + t0;
    for (int e = threadIdx.x; e < nr * opit * NCP; e += blockDim.x) O4[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    const int c0 = P.child_ptr[p], c1 = P.child_ptr[p + 1];
    // the child's part in a z pair: 0 none, 1 first, 2 second
    auto role = [&](int c) -> int {
        if (!PAIR) return 0;
        const int o = Ch.octant[c];
        if (!(o & 1) && c + 1 < c1 && Ch.octant[c + 1] == o + 1) return 1;
        if ((o & 1) && c > c0 && Ch.octant[c - 1] == o - 1) return 2;
        return 0;
    };
    auto fetch_A = [&](int c) {
        const float2 *src = S + ((int64_t)c * 2 + comp) * Kc * Bs + b0 + 2 * pc;
        for (int q = pslot; q < Kc; q += npslot) cp_pair(A4 + q * NCP + pc, src + (int64_t)q * Bs, cols, a16);
    };
    auto fetch_Z = [&](int c) {   // the table of the next phi step: the child's own, or its pair's shift_xy
        const float2 *z = (role(c) ? shift_xy : shift) + (int64_t)Ch.octant[c] * Kp;
        for (int tt = warp; tt < nr; tt += nw)
            for (int u = lane; u < nphp; u += 32) cp8(Z + tt * opit + u, z + tt * nphp + u);
    };
    {
        const WinDev band_t{g1 - g0, wt.tw, wt.start + g0, wt.coef + (size_t)g0 * wt.tw};
        stage_table(band_t, cth, sth);
        stage_table(wp, cph, sph);
        fetch_A(c0);
        cp_commit();
        fetch_Z(c0);
        cp_commit();
    }
    const int cpi = lane % NCP, rl = lane / NCP;
    bool prev_phi = true;   // the previous child ran a phi step (its Z fetch is the newest group)
    for (int c = c0; c < c1; ++c) {
        const int rc = role(c);
        if (prev_phi) cp_wait<1>();   // A(c) (and the tables) are in; Z(c) may still be in flight
        else cp_wait<0>();            // A(c) is the newest group
        __syncthreads();
        // theta: T(t, v) = sum_f c A(row of s + f, v or v + pi); lines v, groups of band rows t
        {
            const int blocks = (nphc + RL - 1) / RL;
            for (Items it(warp, nw, g1 - g0); it.blk < blocks; it.next()) {
                const int gl = it.g, v = it.blk * RL + rl;
                const int vl = min(v, nphc - 1), vr = vl + hc < nphc ? vl + hc : vl + hc - nphc;
                float4 acc[kG];
#pragma unroll
                for (int r = 0; r < kG; ++r) acc[r] = make_float4(0.f, 0.f, 0.f, 0.f);
                win_theta(acc, cth + gl * wt.tw, wt.tw, sth[gl], nthc, A4 + vl * NCP + cpi, A4 + vr * NCP + cpi,
                          nphc * NCP);
                if (v < nphc) {
#pragma unroll
                    for (int r = 0; r < kG; ++r) {
                        const int tt = gl * kG + r;
                        if (tt < nr) {
                            float4 val = acc[r];
                            float4 *t4 = T4 + ((size_t)tt * tpit + v) * NCP + cpi;
                            if (PAIR && rc) {   // scale by the z factor of this child's shift; the second adds
                                const float2 gz = gam[(int64_t)Ch.octant[c] * ntp + tt];
                                val = make_float4(gz.x * val.x - gz.y * val.y, gz.x * val.y + gz.y * val.x,
                                                  gz.x * val.z - gz.y * val.w, gz.x * val.w + gz.y * val.z);
                                if (rc == 2) {
                                    const float4 old = *t4;
                                    val.x += old.x; val.y += old.y; val.z += old.z; val.w += old.w;
                                }
                            }
                            *t4 = val;
                        }
                    }
                }
            }
        }
        __syncthreads();
        if (c + 1 < c1) fetch_A(c + 1);
        cp_commit();
        if (PAIR && rc == 1) {   // the pair's phi step comes with its second child
            prev_phi = false;
            continue;
        }
        cp_wait<1>();   // Z(c) is in; A(c + 1) may still be in flight
        __syncthreads();
        // phi: O(t, u) += Z(t, u) sum_f c T(t, (s + f) mod nphc); lines t, groups of parent phi u
        {
            const int blocks = (nr + RL - 1) / RL;
            for (Items it(warp, nw, wp.groups); it.blk < blocks; it.next()) {
                const int g = it.g, tt = it.blk * RL + rl;
                const int tl = min(tt, nr - 1);
                float4 acc[kG];
#pragma unroll
                for (int r = 0; r < kG; ++r) acc[r] = make_float4(0.f, 0.f, 0.f, 0.f);
                win_periodic<ES>(acc, cph + g * wp.tw, wp.tw, sph[g], nphc, T4 + (size_t)tl * tpit * NCP + cpi);
                if (tt < nr) {
#pragma unroll
                    for (int r = 0; r < kG; ++r) {
                        const int u = g * kG + r;
                        if (u < nphp) {
                            const float2 z = Z[tt * opit + u];
                            float4 *o = O4 + ((size_t)tt * opit + u) * NCP + cpi;
                            float4 y = *o;
                            const float4 a = acc[r];
                            y.x = fmaf(z.x, a.x, fmaf(-z.y, a.y, y.x));
                            y.y = fmaf(z.x, a.y, fmaf(z.y, a.x, y.y));
                            y.z = fmaf(z.x, a.z, fmaf(-z.y, a.w, y.z));
                            y.w = fmaf(z.x, a.w, fmaf(z.y, a.z, y.w));
                            *o = y;
                        }
                    }
                }
            }
        }
        __syncthreads();
        if (c + 1 < c1) fetch_Z(c + 1);
        cp_commit();
        prev_phi = true;
    }
    cp_wait<0>();
    if (!cols) return;
    float2 *dst = reinterpret_cast<float2 *>(P.S) + (((int64_t)p * 2 + comp) * Kp + (int64_t)t0 * nphp) * Bs + b0 + 2 * pc;
    Walk w(pslot, npslot, nphp);
    for (int o = pslot; o < nr * nphp; o += npslot, w.next()) {
        float4 d = O4[(w.t * opit + w.u) * NCP + pc];
        if (accumulate) {
            const float4 y = ld_pair(dst + (int64_t)o * Bs, cols, a16);
            d.x += y.x;
            d.y += y.y;
            d.z += y.z;
            d.w += y.w;
        }
        st_pair(dst + (int64_t)o * Bs, d, cols, a16);
    }
}

constexpr size_t kWinSmemCap = 200 * 1024;

size_t down_win_smem(const DevLevel<float> &P, const DevLevel<float> &Ch, int NB)
{
    return ((size_t)P.nth * (P.nph + 1) + (size_t)P.nth * (Ch.nph + 1)) * NB * sizeof(float2) +
           win_table_bytes(P.wd_ph, P.wd_th);
}

size_t up_win_smem(const DevLevel<float> &P, const DevLevel<float> &Ch, int NB, int RS)
{
    const int gpb = (P.wu_th.groups + RS - 1) / RS;
    const int nr = std::min(P.nth, gpb * kG);
    const WinDev band_t{gpb, P.wu_th.tw, nullptr, nullptr};
    return ((size_t)Ch.K + (size_t)nr * (Ch.nph + 1) + (size_t)nr * (P.nph + 1)) * NB * sizeof(float2) +
           (size_t)nr * (P.nph + 1) * sizeof(float2) + 16 + win_table_bytes(band_t, P.wu_ph);
}

// MINB: CTAs per SM the register budget is set for (3 or 4 for down, 2 or 3 for up)
template <int NB, int MINB, bool PAIR = false>
cudaError_t down_win_nb(const DevLevel<float> &P, const DevLevel<float> &Ch, int B, int Bs, cudaStream_t s)
{
    const size_t smem = down_win_smem(P, Ch, NB);
    if (smem > kWinSmemCap) return cudaErrorInvalidConfiguration;
    if (PAIR && (!P.dgrp || !P.shift_xy || !P.gam)) return cudaErrorInvalidConfiguration;
    dim3 grid((PAIR ? P.ndgrp : Ch.nbox) * ((B + NB - 1) / NB), 2);
    k_down_win<NB, MINB, PAIR><<<grid, 256, smem, s>>>(P, Ch, B, Bs);
    return cudaGetLastError();
}

size_t down_win_pp_smem(const DevLevel<float> &P, const DevLevel<float> &Ch, int NB)
{
    return ((size_t)2 * P.nth * (P.nph + 1) + (size_t)P.nth * (Ch.nph + 1)) * NB * sizeof(float2) +
           win_table_bytes(P.wd_ph, P.wd_th);
}

template <int NB, int MINB>
cudaError_t down_win_pp_nb(const DevLevel<float> &P, const DevLevel<float> &Ch, int B, int Bs, cudaStream_t s)
{
    const size_t smem = down_win_pp_smem(P, Ch, NB);
    if (smem > kWinSmemCap) return cudaErrorInvalidConfiguration;
    dim3 grid(P.nbox * ((B + NB - 1) / NB), 2);
    k_down_win_pp<NB, MINB><<<grid, 256, smem, s>>>(P, Ch, B, Bs);
    return cudaGetLastError();
}

template <int NB, int MINB, bool PAIR = false>
cudaError_t up_win_nb(const DevLevel<float> &P, const DevLevel<float> &Ch, int B, int Bs, int acc, cudaStream_t s)
{
    if (PAIR && (!P.shift_xy || !P.gam)) return cudaErrorInvalidConfiguration;
    // bands of parent theta groups: shared memory for MINB CTAs per SM, and
    // enough CTAs to fill the GPU
    const size_t cap = (size_t)(MINB >= 3 ? 72 : 100) * 1024;
    int RS = 1;
    while (RS < P.wu_th.groups && up_win_smem(P, Ch, NB, RS) > cap) ++RS;
    const int64_t ctas = (int64_t)P.nbox * 2 * ((B + NB - 1) / NB);
    while (ctas * RS < 4 * 152 && 2 * RS <= P.wu_th.groups) RS *= 2;
    const size_t smem = up_win_smem(P, Ch, NB, RS);
    if (smem > kWinSmemCap) return cudaErrorInvalidConfiguration;
    dim3 grid(P.nbox * ((B + NB - 1) / NB) * RS, 2);
    k_up_win<NB, MINB, PAIR><<<grid, 256, smem, s>>>(P, Ch, B, RS, Bs, acc);
    return cudaGetLastError();
}

bool win_ok(const WinDev &a, const WinDev &b) { return a.groups > 0 && b.groups > 0 && a.coef && b.coef; }

}  // namespace

cudaError_t launch_down_win(const DevLevel<float> &P, const DevLevel<float> &Ch, int B, int Bs, int nb,
                            cudaStream_t s)
{
    if (!win_ok(P.wd_ph, P.wd_th) || B < 1) return cudaErrorInvalidConfiguration;
    switch (nb) {
    case 4: return down_win_nb<4, 3>(P, Ch, B, Bs, s);
    case 8: return down_win_nb<8, 3>(P, Ch, B, Bs, s);
    case 16: return down_win_nb<16, 3>(P, Ch, B, Bs, s);
    case 104: return down_win_nb<4, 4>(P, Ch, B, Bs, s);
    case 108: return down_win_nb<8, 4>(P, Ch, B, Bs, s);
    case 504: return down_win_nb<4, 3, true>(P, Ch, B, Bs, s);
    case 508: return down_win_nb<8, 3, true>(P, Ch, B, Bs, s);
    case 204: return down_win_pp_nb<4, 3>(P, Ch, B, Bs, s);
    case 208: return down_win_pp_nb<8, 2>(P, Ch, B, Bs, s);
    default: return cudaErrorInvalidConfiguration;
    }
}

cudaError_t launch_up_win(const DevLevel<float> &P, const DevLevel<float> &Ch, int B, int Bs, int acc, int nb,
                          cudaStream_t s)
{
    if (!win_ok(P.wu_th, P.wu_ph) || B < 1) return cudaErrorInvalidConfiguration;
    switch (nb) {
    case 4: return up_win_nb<4, 2>(P, Ch, B, Bs, acc, s);
    case 8: return up_win_nb<8, 2>(P, Ch, B, Bs, acc, s);
    case 16: return up_win_nb<16, 2>(P, Ch, B, Bs, acc, s);
    case 104: return up_win_nb<4, 3>(P, Ch, B, Bs, acc, s);
    case 108: return up_win_nb<8, 3>(P, Ch, B, Bs, acc, s);
    case 404: return up_win_nb<4, 2, true>(P, Ch, B, Bs, acc, s);
    case 408: return up_win_nb<8, 2, true>(P, Ch, B, Bs, acc, s);
    case 416: return up_win_nb<16, 2, true>(P, Ch, B, Bs, acc, s);
    default: return cudaErrorInvalidConfiguration;
    }
}

cudaError_t prime_win_kernels()
{
    cudaError_t e;
#define ALLOW(k) do { if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWinSmemCap)) != cudaSuccess) return e; } while (0)
    ALLOW((k_down_win<4, 3>)); ALLOW((k_down_win<8, 3>)); ALLOW((k_down_win<16, 3>));
    ALLOW((k_down_win<4, 4>)); ALLOW((k_down_win<8, 4>));
    ALLOW((k_down_win_pp<4, 3>)); ALLOW((k_down_win_pp<8, 2>));
    ALLOW((k_down_win<4, 3, true>)); ALLOW((k_down_win<8, 3, true>));
    ALLOW((k_up_win<4, 2>)); ALLOW((k_up_win<8, 2>)); ALLOW((k_up_win<16, 2>));
    ALLOW((k_up_win<4, 3>)); ALLOW((k_up_win<8, 3>));
    ALLOW((k_up_win<4, 2, true>)); ALLOW((k_up_win<8, 2, true>)); ALLOW((k_up_win<16, 2, true>));
#undef ALLOW
    return cudaSuccess;
}

}  // namespace mlfma
