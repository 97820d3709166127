// Local Lagrange interpolation (upward pass) and anterpolation (downward
// pass) of Section III-C on the fifth-generation tensor cores: tcgen05.mma
// kind::tf32 with the accumulators in tensor memory.
//
// Both steps of the separable interpolation are dense products once the
// columns are batched: a CTA takes one parent (up) or child (down) box, one
// field component and chunks of 4 complex columns, so every sample of the
// field is 8 real rows (column, re/im) of the M = 128 operand tiles.
//
//   up    (child level -> parent level), per child:
//         step 1, phi:   T[(thc, b, ri)][php] = sum_phc S[thc][phc] Phi[php][phc]
//         step 2, theta: U[(php, b, ri)][thp] = sum_thc T[thc][php] Th[thp][thc]
//                                             + sum_thc T[thc][php + pi] Thr[thp][thc]
//         S_parent[thp][php] += shift_child[thp][php] U           (accumulated in TMEM)
//   down  (parent level -> child level):
//         Y = conj(shift_child) G_parent
//         step 1, theta: V[(php, b, ri)][thc] = sum_thp Y[thp][php] ThD[thc][thp]
//                                             + sum_thp Y[thp][php + pi] ThDr[thc][thp]
//         step 2, phi:   G_child[thc][phc] += sum_php V[thc][php] PhD[phc][php]
//
// The up pass is phi then theta and the down pass its exact transpose
// (theta then phi) with the weights folded into the anterpolation matrices,
// so anterpolation stays the weighted transpose of interpolation.  The
// samples at phi + pi that theta stencils reach across the poles form a
// second block of K columns (kr0 on) whose matrix carries the sign flip.
//
// Operands: A tiles are written by the threads into shared memory in the
// K-major 128-byte-swizzled layout (8-row groups of 1024 bytes, 32 TF32
// values per row and K-atom); the threads of a warp cover 8 consecutive
// rows x 4 consecutive K, which makes every 4-byte store conflict-free.  B
// operands (the interpolation matrices) are prepared on the host in the
// same layout and copied in once per CTA.  One thread issues the MMAs and
// commits them to an mbarrier; the tensor-memory results are read with
// tcgen05.ld 32x32b (thread = row).  SPLIT: 3xTF32 (A_hi B_hi + A_hi B_lo +
// A_lo B_hi, hi = the FP32 value rounded to the nearest TF32), accurate to
// FP32 rounding; otherwise one TF32 product of the rounded operands.
//
// Every wait is bounded: a wait that runs out sets *um_err, skips the rest
// of the work, waits (bounded) for MMAs in flight, frees the tensor memory
// and returns.  A test hook (um_test, set from the environment variable
// MLFMA_TEST_WITHHOLD_ARRIVAL when the plan is made) has the first CTA of
// every launch issue nothing for its first step, so that its wait runs out.
#include "device.h"

#include <algorithm>
#include <cstdint>

namespace mlfma {

namespace {

constexpr int kTile = 128;          // rows of an A tile
constexpr int kCols = 4;            // complex columns per chunk
constexpr int kTileBytesPerAtom = kTile * 128;
constexpr long long kWaitPolls = 1ll << 24;
constexpr long long kTestPolls = 1ll << 12;   // the test hook's shortened wait

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO), version 1
__device__ __forceinline__ uint64_t sdesc(uint32_t addr)
{
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// instruction descriptor: D FP32, A and B TF32, both K-major, M = 128
__device__ __forceinline__ uint32_t idesc(int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kTile >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc)
{
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d),
                 "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar)));
}

__device__ __forceinline__ bool wait_bar(uint64_t *bar, uint32_t parity, long long polls)
{
    uint32_t done = 0;
    for (long long it = 0; it < polls && !done; ++it)
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done)
                     : "r"(su32(bar)), "r"(parity));
    return done != 0;
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's tensor-memory lane
__device__ __forceinline__ void tld16(uint32_t addr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15])
                 : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tst16(uint32_t addr, const float (&v)[16])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
                 ::"r"(addr), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                 "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                 "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
                 "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
                 "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
                 "r"(__float_as_uint(v[15])));
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// byte offset of element (r, k) in a K-major swizzled operand of R rows
__device__ __forceinline__ uint32_t kmaj(int r, int k, int R)
{
    return (uint32_t)((k >> 5) * (R << 7) + (r >> 3) * 1024 + (r & 7) * 128 + ((((k & 31) >> 2) ^ (r & 7)) << 4) +
                      ((k & 3) << 2));
}

// FP32 -> nearest TF32 (10 mantissa bits), ties away from zero: add half a
// TF32 unit in the last place to the magnitude bits and clear the 13 low
// bits.  The tensor cores read an operand's top 19 bits, so a value rounded
// here is taken exactly; left to the hardware it would be truncated, and
// truncation errors all point towards zero and add up.
__device__ __forceinline__ float tf32_rn(float v)
{
    return __uint_as_float((__float_as_uint(v) + 0x1000u) & 0xFFFFE000u);
}

// store one A element: hi = nearest TF32 and, with SPLIT, lo = v - hi (exact
// in FP32)
template <bool SPLIT>
__device__ __forceinline__ void put(unsigned char *hi, unsigned char *lo, uint32_t off, float v)
{
    const float h = tf32_rn(v);
    *reinterpret_cast<float *>(hi + off) = h;
    if (SPLIT) *reinterpret_cast<float *>(lo + off) = v - h;
}

// All MMAs of one step into tensor-memory columns d: A tile (hi, lo) x the
// step's matrix (hi, lo), skipping K-steps whose coefficients are all zero.
template <bool SPLIT>
__device__ __forceinline__ void issue(uint32_t d, uint32_t ah, uint32_t al, uint32_t bh, uint32_t bl, const UmmaStep &st)
{
    const uint32_t id = idesc(st.N);
    uint32_t acc = 0;
    for (int s = 0; s < st.K / 8; ++s) {
        if (!((st.kmask >> s) & 1u)) continue;
        const uint32_t ao = (uint32_t)((s >> 2) * kTileBytesPerAtom + (s & 3) * 32);
        const uint32_t bo = (uint32_t)((s >> 2) * (st.N << 7) + (s & 3) * 32);
        if (SPLIT) {
            mma(d, sdesc(al + ao), sdesc(bh + bo), id, acc);
            acc = 1;
            mma(d, sdesc(ah + ao), sdesc(bl + bo), id, acc);
        }
        mma(d, sdesc(ah + ao), sdesc(bh + bo), id, acc);
        acc = 1;
    }
}

__host__ __device__ __forceinline__ int atoms(int K) { return (K + 31) >> 5; }

__device__ __forceinline__ unsigned char *align1024(unsigned char *p)
{
    return reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(p) + 1023) & ~(uintptr_t)1023);
}

// Tensor-memory columns to allocate: a power of two >= 32.
__host__ __device__ inline int tmem_cols(int need)
{
    int c = 32;
    while (c < need) c <<= 1;
    return c;
}

// Asynchronous global -> shared copies of 8 bytes (one complex FP32 value),
// in commit groups.
__device__ __forceinline__ void cp8(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(su32(dst)), "l"(src));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Copy columns [b0, b0 + 4) of samples [0, K) of one field block (rows of Bs
// complex values) into raw[q * pitch + c] (8 floats per sample: 4 columns x
// re/im); columns at or beyond B are zero.  pitch counts floats per sample
// row group: raw row of sample q starts at (q / nph) * rowp + (q % nph) * 8.
__device__ __forceinline__ void stage_field(float *raw, const float *src, int K, int nph, int rowp, int Bs, int b0, int B)
{
    for (int e = threadIdx.x; e < K * kCols; e += blockDim.x) {
        const int q = e >> 2, c = e & 3;
        float *d = raw + (q / nph) * rowp + (q % nph) * 8 + c * 2;
        if (b0 + c < B) {
            cp8(d, src + ((size_t)q * Bs + b0 + c) * 2);
        } else {
            d[0] = 0.0f;
            d[1] = 0.0f;
        }
    }
}

// The tensor-memory allocation, operand images and the shared A tile buffer
// (steps 1 and 2 never hold it at the same time).
struct Ctx {
    unsigned char *b1h, *b1l, *b2h, *b2l, *ah, *al, *rest;
    uint32_t tmem;
};

template <bool SPLIT>
__device__ void setup(Ctx &c, unsigned char *sm, const unsigned char *img, int img_bytes, const UmmaStep &s1,
                      const UmmaStep &s2, uint64_t *bar, uint32_t *tslot, int ncols)
{
    const int tid = threadIdx.x;
    c.b1h = sm + s1.off;
    c.b1l = c.b1h + s1.bytes;
    c.b2h = sm + s2.off;
    c.b2l = c.b2h + s2.bytes;
    const int abytes = max(atoms(s1.K), atoms(s2.K)) * kTileBytesPerAtom;
    c.ah = sm + ((img_bytes + 1023) & ~1023);
    c.al = SPLIT ? c.ah + abytes : c.ah;
    c.rest = c.ah + (SPLIT ? 2 : 1) * abytes;
    const uint4 *src = reinterpret_cast<const uint4 *>(img);
    uint4 *dst = reinterpret_cast<uint4 *>(sm);
    for (int i = tid; i < img_bytes / 16; i += blockDim.x) dst[i] = src[i];
    // A tiles start at zero; afterwards every value in them is finite, and
    // padding columns meet zero coefficients
    uint4 *z = reinterpret_cast<uint4 *>(c.ah);
    const int nz = (int)((c.rest - c.ah) / 16);
    for (int i = tid; i < nz; i += blockDim.x) z[i] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(bar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (tid < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    c.tmem = *tslot;
}

__device__ __forceinline__ void teardown(uint32_t tmem, int ncols)
{
    fence_before();
    __syncthreads();
    fence_after();
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

// Make this step's A tile visible to the tensor cores, issue its MMAs from
// one thread and wait for them; false when the wait ran out.  withhold (a
// test hook): issue nothing, so that nothing arrives and the (shortened)
// wait runs out.
template <bool SPLIT>
__device__ __forceinline__ bool run_step(uint32_t d, const Ctx &c, bool second, const UmmaStep &st, uint64_t *bar,
                                         uint32_t &phase, bool withhold)
{
    fence_async_smem();
    fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && !withhold) {
        fence_after();
        issue<SPLIT>(d, su32(c.ah), su32(c.al), su32(second ? c.b2h : c.b1h), su32(second ? c.b2l : c.b1l), st);
        commit(bar);
    }
    const bool ok = wait_bar(bar, phase, withhold ? kTestPolls : kWaitPolls);
    phase ^= 1u;
    fence_after();
    return __syncthreads_and(ok);
}

__device__ __forceinline__ void sync_tmem()
{
    fence_before();
    __syncthreads();
    fence_after();
}

// ------------------------------------------------------------------- up ---
// grid (parent box, component, column-chunk group); 128 threads.  The work
// items are (chunk, child) pairs; the next item's child field is copied in
// (cp.async) while the current one is interpolated, and each phi tile's
// phase shifts while its MMAs run.
template <bool SPLIT>
__global__ void __launch_bounds__(128) k_up_umma(DevLevel<float> P, DevLevel<float> Ch, int B, int Bs, int accumulate,
                                                 int cpc)
{
    extern __shared__ unsigned char smraw[];
    __shared__ uint64_t bar;
    __shared__ uint32_t tslot;
    unsigned char *sm = align1024(smraw);
    const UmmaStep s1 = P.um_up1, s2 = P.um_up2;
    const int tiles1 = (Ch.nth + 15) / 16, tiles2 = (P.nph + 15) / 16;
    const int cD1 = 0, cD2 = tiles1 * s1.N, cAcc = cD2 + s2.N;
    const int ncols = tmem_cols(cAcc + tiles2 * s2.N);
    Ctx c;
    setup<SPLIT>(c, sm, P.um_up, P.um_up_bytes, s1, s2, &bar, &tslot, ncols);
    const int Kc = Ch.K;
    float *const raw0 = reinterpret_cast<float *>(c.rest);   // two buffers of Kc samples x 8 floats
    auto raw = [&](int i) { return raw0 + (size_t)(i & 1) * Kc * 8; };
    float2 *sb = reinterpret_cast<float2 *>(c.rest + (size_t)2 * Kc * 32);   // [N2][16] phase shifts of a phi tile
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t lanes = (uint32_t)(warp * 32) << 16;
    const int p = blockIdx.x, comp = blockIdx.y;
    const int ch0 = P.child_ptr[p], nch = P.child_ptr[p + 1] - ch0;
    const int nthc = Ch.nth, nphc = Ch.nph, nthp = P.nth, nphp = P.nph, hp = nphp / 2;
    const int rsub = lane & 7, klo = lane >> 3, bcol = rsub >> 1, ri = lane & 1;
    const bool withhold = P.um_test && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0;
    const int chunk0 = blockIdx.z * cpc;
    const int nchunk = max(0, min(cpc, (B + kCols - 1) / kCols - chunk0));
    const int nitems = nchunk * nch;
    auto stage_item = [&](int it, float *dst) {
        const int ci = it / nch, chd = ch0 + it % nch;
        stage_field(dst, Ch.S + ((size_t)(chd * 2 + comp) * Kc) * Bs * 2, Kc, nphc, nphc * 8, Bs,
                    (chunk0 + ci) * kCols, B);
    };
    if (nitems > 0) stage_item(0, raw(0));
    cp_commit();
    uint32_t phase = 0;
    bool ok = true;
    for (int it = 0; it < nitems && ok; ++it) {
        const int ci = it / nch, chd = ch0 + it % nch;
        const bool first = it % nch == 0, last = it % nch == nch - 1;
        const int b0 = (chunk0 + ci) * kCols;
        const bool bok = b0 + bcol < B;
        if (it + 1 < nitems) stage_item(it + 1, raw(it + 1));
        cp_commit();
        cp_wait<1>();
        __syncthreads();
        const float *r = raw(it);
        // step 1 (phi), tile by tile of child theta rows
        for (int t1 = 0; t1 < tiles1 && ok; ++t1) {
            for (int g = warp; g < 16 * (s1.K / 4); g += 4) {
                const int rg = g & 15, k = (g >> 4) * 4 + klo;
                const int thc = t1 * 16 + rg;
                const float v = (thc < nthc && k < nphc) ? r[(thc * nphc + k) * 8 + rsub] : 0.0f;
                put<SPLIT>(c.ah, c.al, kmaj(rg * 8 + rsub, k, kTile), v);
            }
            ok = run_step<SPLIT>(c.tmem + cD1 + t1 * s1.N, c, false, s1, &bar, phase, withhold);
        }
        if (!ok) break;
        // step 2 (theta), tile by tile of parent phi samples
        const float2 *sh = reinterpret_cast<const float2 *>(P.shift) + (size_t)Ch.octant[chd] * P.K;
        for (int t2 = 0; t2 < tiles2 && ok; ++t2) {
            const int php0 = t2 * 16, phr0 = (php0 + hp) % nphp;
            for (int e = tid; e < s2.N * 16; e += blockDim.x) {
                const int thp = e >> 4, j = e & 15;
                if (thp < nthp && php0 + j < nphp) cp8(sb + e, sh + thp * nphp + php0 + j);
                else sb[e] = make_float2(0.0f, 0.0f);
            }
            cp_commit();
            for (int t1 = 0; t1 < tiles1; ++t1) {
                const int thc = t1 * 16 + warp * 4 + klo;
                float v[16];
                tld16(c.tmem + lanes + cD1 + t1 * s1.N + php0, v);
                if (thc < nthc) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) put<SPLIT>(c.ah, c.al, kmaj(i * 8 + rsub, thc, kTile), v[i]);
                }
                const int kr = s2.kr0 + thc;
                const bool need = thc < nthc && ((s2.kmask >> (kr >> 3)) & 1u);
                if (__any_sync(0xffffffffu, need)) {
                    tld16(c.tmem + lanes + cD1 + t1 * s1.N + phr0, v);
                    if (need) {
#pragma unroll
                        for (int i = 0; i < 16; ++i) put<SPLIT>(c.ah, c.al, kmaj(i * 8 + rsub, kr, kTile), v[i]);
                    }
                }
            }
            ok = run_step<SPLIT>(c.tmem + cD2, c, true, s2, &bar, phase, false);
            if (!ok) break;
            cp_wait<0>();
            __syncthreads();
            // shift and accumulate: this thread's row is (php, column, re/im)
            const int pl = warp * 4 + klo;
            for (int n0 = 0; n0 < s2.N; n0 += 16) {
                float v[16], a[16];
                tld16(c.tmem + lanes + cD2 + n0, v);
                if (first) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) a[i] = 0.0f;
                } else {
                    tld16(c.tmem + lanes + cAcc + t2 * s2.N + n0, a);
                }
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const float o = __shfl_xor_sync(0xffffffffu, v[i], 1);
                    const float re = ri ? o : v[i], im = ri ? v[i] : o;
                    const float2 z = sb[(n0 + i) * 16 + pl];
                    a[i] += ri ? (z.x * im + z.y * re) : (z.x * re - z.y * im);
                }
                tst16(c.tmem + lanes + cAcc + t2 * s2.N + n0, a);
            }
            sync_tmem();
        }
        if (!ok || !last) continue;
        // the parent field of this chunk
        float *dst = P.S + ((size_t)(p * 2 + comp) * P.K) * Bs * 2;
        for (int t2 = 0; t2 < tiles2; ++t2) {
            const int php = t2 * 16 + warp * 4 + klo;
            for (int n0 = 0; n0 < s2.N; n0 += 16) {
                float a[16];
                tld16(c.tmem + lanes + cAcc + t2 * s2.N + n0, a);
                if (php < nphp && bok) {
                    float old[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int thp = n0 + i;
                        old[i] = (accumulate && thp < nthp) ? dst[((size_t)(thp * nphp + php) * Bs + b0 + bcol) * 2 + ri]
                                                            : 0.0f;
                    }
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int thp = n0 + i;
                        if (thp < nthp) dst[((size_t)(thp * nphp + php) * Bs + b0 + bcol) * 2 + ri] = old[i] + a[i];
                    }
                }
            }
        }
        sync_tmem();
    }
    cp_wait<0>();
    if (!ok) {
        if (tid == 0) atomicExch(P.um_err, 1);
        // an MMA group may still be in flight: give it a bounded time to land
        wait_bar(&bar, phase, withhold ? kTestPolls : kWaitPolls);
    }
    teardown(c.tmem, ncols);
}

// ----------------------------------------------------------------- down ---
// grid (child box, component, column-chunk group); 128 threads.  The
// child's phase shifts are copied in once; the parent field of each column
// chunk is copied in (cp.async) ahead of its use: the next chunk's while this
// one is worked on (nbuf = 2), or during this one's second step (nbuf = 1).
// The parent field rows (one theta) are padded by one sample so that a warp
// reading four theta rows of one phi hits distinct banks.
template <bool SPLIT>
__global__ void __launch_bounds__(128) k_down_umma(DevLevel<float> P, DevLevel<float> Ch, int B, int Bs, int cpc,
                                                   int nbuf)
{
    extern __shared__ unsigned char smraw[];
    __shared__ uint64_t bar;
    __shared__ uint32_t tslot;
    unsigned char *sm = align1024(smraw);
    const UmmaStep s1 = P.um_dn1, s2 = P.um_dn2;
    const int tiles1 = (P.nph + 15) / 16, tiles2 = (Ch.nth + 15) / 16;
    const int cD1 = 0, cD2 = tiles1 * s1.N;
    const int ncols = tmem_cols(cD2 + s2.N);
    Ctx c;
    setup<SPLIT>(c, sm, P.um_dn, P.um_dn_bytes, s1, s2, &bar, &tslot, ncols);
    const int Kp = P.K, nthc = Ch.nth, nphc = Ch.nph, nthp = P.nth, nphp = P.nph, hp = nphp / 2;
    const int rowp = (nphp + 1) * 8;                       // floats per parent theta row in shared memory
    float2 *shs = reinterpret_cast<float2 *>(c.rest);      // [Kp] this child's phase shifts
    float *const raw0 = reinterpret_cast<float *>(c.rest + (size_t)Kp * 8);
    auto raw = [&](int i) { return raw0 + (size_t)(i & 1) * nthp * rowp; };
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t lanes = (uint32_t)(warp * 32) << 16;
    const int chd = blockIdx.x, comp = blockIdx.y;
    const int par = Ch.parent[chd], oct = Ch.octant[chd];
    const int rsub = lane & 7, klo = lane >> 3, bcol = rsub >> 1, ri = lane & 1;
    const float *g = P.G + ((size_t)(par * 2 + comp) * Kp) * Bs * 2;
    const float2 *sh = reinterpret_cast<const float2 *>(P.shift) + (size_t)oct * Kp;
    float *dst = Ch.G + ((size_t)(chd * 2 + comp) * Ch.K) * Bs * 2;
    const bool withhold = P.um_test && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0;
    const int chunk0 = blockIdx.z * cpc;
    const int nchunk = max(0, min(cpc, (B + kCols - 1) / kCols - chunk0));
    for (int q = tid; q < Kp; q += blockDim.x) cp8(shs + q, sh + q);
    if (nchunk > 0) stage_field(raw(0), g, Kp, nphp, rowp, Bs, chunk0 * kCols, B);
    cp_commit();
    uint32_t phase = 0;
    bool ok = true;
    for (int ci = 0; ci < nchunk && ok; ++ci) {
        const int b0 = (chunk0 + ci) * kCols;
        const bool bok = b0 + bcol < B;
        const float *r = raw(nbuf == 2 ? ci : 0);
        if (nbuf == 2 && ci + 1 < nchunk) stage_field(raw(ci + 1), g, Kp, nphp, rowp, Bs, b0 + kCols, B);
        cp_commit();
        cp_wait<1>();
        __syncthreads();
        // step 1 (theta), tile by tile of parent phi samples: rows (php, column, re/im)
        for (int t1 = 0; t1 < tiles1 && ok; ++t1) {
            for (int gi = warp; gi < 16 * (s1.K / 4); gi += 4) {
                const int rg = gi & 15, k = (gi >> 4) * 4 + klo;
                const int php = t1 * 16 + rg;
                int thp = -1, ph = php;
                if (k < nthp) thp = k;
                else if (k >= s1.kr0 && k < s1.kr0 + nthp) { thp = k - s1.kr0; ph = (php + hp) % nphp; }
                float v = 0.0f;
                if (thp >= 0 && php < nphp && ((s1.kmask >> (k >> 3)) & 1u)) {
                    const float *x = r + thp * rowp + ph * 8 + bcol * 2;
                    const float2 z = shs[thp * nphp + ph];
                    // conj(z) (re + i im)
                    v = ri ? (z.x * x[1] - z.y * x[0]) : (z.x * x[0] + z.y * x[1]);
                }
                put<SPLIT>(c.ah, c.al, kmaj(rg * 8 + rsub, k, kTile), v);
            }
            ok = run_step<SPLIT>(c.tmem + cD1 + t1 * s1.N, c, false, s1, &bar, phase, withhold);
        }
        if (!ok) break;
        if (nbuf == 1 && ci + 1 < nchunk) {   // the parent field of this chunk is no longer needed
            __syncthreads();
            stage_field(raw(0), g, Kp, nphp, rowp, Bs, b0 + kCols, B);
            cp_commit();
        }
        // step 2 (phi), tile by tile of child theta rows
        for (int t2 = 0; t2 < tiles2 && ok; ++t2) {
            for (int t1 = 0; t1 < tiles1; ++t1) {
                const int php = t1 * 16 + warp * 4 + klo;
                float v[16];
                tld16(c.tmem + lanes + cD1 + t1 * s1.N + t2 * 16, v);
                if (php < s2.K) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) put<SPLIT>(c.ah, c.al, kmaj(i * 8 + rsub, php, kTile), v[i]);
                }
            }
            ok = run_step<SPLIT>(c.tmem + cD2, c, true, s2, &bar, phase, false);
            if (!ok) break;
            const int thc = t2 * 16 + warp * 4 + klo;
            for (int n0 = 0; n0 < s2.N; n0 += 16) {
                float v[16];
                tld16(c.tmem + lanes + cD2 + n0, v);
                if (thc < nthc && bok) {
                    float old[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int phc = n0 + i;
                        old[i] = phc < nphc ? dst[((size_t)(thc * nphc + phc) * Bs + b0 + bcol) * 2 + ri] : 0.0f;
                    }
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int phc = n0 + i;
                        if (phc < nphc) dst[((size_t)(thc * nphc + phc) * Bs + b0 + bcol) * 2 + ri] = old[i] + v[i];
                    }
                }
            }
            sync_tmem();
        }
    }
    cp_wait<0>();
    if (!ok) {
        if (tid == 0) atomicExch(P.um_err, 1);
        wait_bar(&bar, phase, withhold ? kTestPolls : kWaitPolls);
    }
    teardown(c.tmem, ncols);
}

template <bool SPLIT>
size_t umma_smem(int img_bytes, const UmmaStep &s1, const UmmaStep &s2, size_t rest)
{
    const size_t a = (size_t)std::max(atoms(s1.K), atoms(s2.K)) * kTileBytesPerAtom * (SPLIT ? 2 : 1);
    return ((size_t)img_bytes + 1023) / 1024 * 1024 + a + rest + 1024;
}

constexpr size_t kUmmaSmemCap = 220 * 1024;

template <class K>
cudaError_t allow(K k, size_t smem)
{
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// Column-chunk groups per CTA: enough CTAs for a few per SM, fewer set-ups.
int chunks_per_cta(int64_t boxes, int B)
{
    const int chunks = (B + kCols - 1) / kCols;
    int cpc = 1;
    while (cpc * 2 <= chunks && boxes * 2 * ((chunks + cpc * 2 - 1) / (cpc * 2)) >= 152 * 6) cpc *= 2;
    return cpc;
}

}  // namespace

// Tensor-core up pass from level l+1 into level l (P = level l).  Returns
// cudaErrorInvalidConfiguration, launching nothing, when the level has no
// tensor-core tables or its operands do not fit.
cudaError_t launch_up_umma(const DevLevel<float> &P, const DevLevel<float> &Ch, int B, int Bs, int acc, bool split,
                           cudaStream_t s)
{
    if (!P.um_up || !P.um_err) return cudaErrorInvalidConfiguration;
    const size_t rest = (size_t)2 * Ch.K * 32 + (size_t)P.um_up2.N * 16 * 8;
    const size_t smem = split ? umma_smem<true>(P.um_up_bytes, P.um_up1, P.um_up2, rest)
                              : umma_smem<false>(P.um_up_bytes, P.um_up1, P.um_up2, rest);
    if (smem > kUmmaSmemCap) return cudaErrorInvalidConfiguration;
    const int cpc = chunks_per_cta(P.nbox, B);
    const int chunks = (B + kCols - 1) / kCols;
    dim3 grid(P.nbox, 2, (chunks + cpc - 1) / cpc);
    cudaError_t e;
    if (split) {
        if ((e = allow(k_up_umma<true>, smem)) != cudaSuccess) return e;
        k_up_umma<true><<<grid, 128, smem, s>>>(P, Ch, B, Bs, acc, cpc);
    } else {
        if ((e = allow(k_up_umma<false>, smem)) != cudaSuccess) return e;
        k_up_umma<false><<<grid, 128, smem, s>>>(P, Ch, B, Bs, acc, cpc);
    }
    return cudaGetLastError();
}

// Tensor-core down pass from level l (P) into level l+1 (Ch), added into the
// child's incoming field.  Same refusal rule as launch_up_umma.
cudaError_t launch_down_umma(const DevLevel<float> &P, const DevLevel<float> &Ch, int B, int Bs, bool split,
                             cudaStream_t s)
{
    if (!P.um_dn || !P.um_err) return cudaErrorInvalidConfiguration;
    const size_t one = (size_t)P.nth * (P.nph + 1) * 32;
    auto need = [&](int nbuf) {
        const size_t rest = (size_t)P.K * 8 + nbuf * one;
        return split ? umma_smem<true>(P.um_dn_bytes, P.um_dn1, P.um_dn2, rest)
                     : umma_smem<false>(P.um_dn_bytes, P.um_dn1, P.um_dn2, rest);
    };
    // double-buffer only while two CTAs still fit on an SM
    const int nbuf = need(2) <= kUmmaSmemCap / 2 ? 2 : 1;
    const size_t smem = need(nbuf);
    if (smem > kUmmaSmemCap) return cudaErrorInvalidConfiguration;
    const int cpc = chunks_per_cta(Ch.nbox, B);
    const int chunks = (B + kCols - 1) / kCols;
    dim3 grid(Ch.nbox, 2, (chunks + cpc - 1) / cpc);
    cudaError_t e;
    if (split) {
        if ((e = allow(k_down_umma<true>, smem)) != cudaSuccess) return e;
        k_down_umma<true><<<grid, 128, smem, s>>>(P, Ch, B, Bs, cpc, nbuf);
    } else {
        if ((e = allow(k_down_umma<false>, smem)) != cudaSuccess) return e;
        k_down_umma<false><<<grid, 128, smem, s>>>(P, Ch, B, Bs, cpc, nbuf);
    }
    return cudaGetLastError();
}

}  // namespace mlfma
