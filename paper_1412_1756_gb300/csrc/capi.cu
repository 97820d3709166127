// C ABI (include/mlfma.h): plan construction, products, inspection.
#include "../../include/mlfma.h"
#include "device.h"
#include "plan_host.h"

#include <algorithm>
#include <chrono>
#include <complex>
#include <cmath>
#include <cstring>
#include <cstdlib>
#include <map>
#include <memory>
#include <new>
#include <string>
#include <vector>

using namespace mlfma;

namespace {

thread_local std::string g_err;

mlfma_status fail(mlfma_status st, const std::string &msg)
{
    g_err = msg;
    return st;
}

mlfma_status cuda_fail(cudaError_t e, const char *where)
{
    g_err = std::string(where) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? MLFMA_ENOMEM : MLFMA_ECUDA;
}

struct DevMem {
    std::vector<void *> ptrs;
    int64_t bytes = 0;
    cudaError_t alloc(void **p, size_t n)
    {
        *p = nullptr;
        if (n == 0) n = 16;
        cudaError_t e = cudaMalloc(p, n);
        if (e == cudaSuccess) {
            ptrs.push_back(*p);
            bytes += (int64_t)n;
        }
        return e;
    }
    template <class T>
    cudaError_t upload(const T *src, size_t count, const T **out)
    {
        void *p;
        cudaError_t e = alloc(&p, count * sizeof(T));
        if (e != cudaSuccess) return e;
        if (count) e = cudaMemcpy(p, src, count * sizeof(T), cudaMemcpyHostToDevice);
        *out = static_cast<const T *>(p);
        return e;
    }
    template <class T>
    cudaError_t upload(const std::vector<T> &v, const T **out) { return upload(v.data(), v.size(), out); }
    void release(void *p)
    {
        for (auto &q : ptrs)
            if (q == p) {
                cudaFree(q);
                q = nullptr;
            }
    }
    void free_all()
    {
        for (void *p : ptrs)
            if (p) cudaFree(p);
        ptrs.clear();
    }
};

class DeviceGuard {
  public:
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&prev_);
        if (dev >= 0 && dev != prev_) {
            cudaSetDevice(dev);
            set_ = true;
        }
    }
    ~DeviceGuard()
    {
        if (set_) cudaSetDevice(prev_);
    }

  private:
    int prev_ = 0;
    bool set_ = false;
};

}  // namespace

struct mlfma_plan_s {
    PlanHost host;
    mlfma_opts opts{};
    int device = -1;
    bool on_device = false;
    DevMem mem;
    ProductArgs<float> a32;
    ProductArgs<double> a64;
    bool has32 = false, has64 = false;
    void *stage_x = nullptr, *stage_y = nullptr;   // host-API staging (largest type)
    double setup_seconds = 0;
    CoreStreams cs;                                  // plan-owned streams/events of the core pass
    std::map<std::pair<int, int>, cudaGraphExec_t> graphs;   // (precision, columns) -> captured core
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;   // caller stream <-> plan streams
    StageClock clock;
    // FP64 setup inputs kept for the derivative tables, built on first use
    DevMesh dm;
    const int32_t *d_ubox = nullptr;
    const double *d_grid = nullptr, *d_bc = nullptr;
    bool dk_ready[2] = {false, false};   // per precision
    // products of the paper's kernel variants (Section IV): X u by the
    // cos(kR)/R kernel (Eq. (XI)) and R u by the sin(kR)/R kernel with
    // sibling translations (Eq. (RI)), set up on first use per precision
    ProductArgs<float> ax32, ar32;
    ProductArgs<double> ax64, ar64;
    bool x_ready[2] = {false, false}, r_ready[2] = {false, false};
    std::map<std::pair<int, int>, Tuning> tunes;   // (precision, internal columns) -> launch choices
};

namespace {

constexpr int kIntSlots = 22;   // device integer tables per level

template <class R>
cudaError_t upload_pairs(DevMem &M, const std::vector<cd> &v, const R **out)
{
    std::vector<R> t(2 * v.size());
    for (size_t i = 0; i < v.size(); ++i) { t[2 * i] = (R)v[i].real(); t[2 * i + 1] = (R)v[i].imag(); }
    return M.upload(t, out);
}

// Tables of a parent level l (to and from level l + 1): phase shifts, the
// packed interpolation stencils and the anterpolation stencils zero-padded
// to dn_taps taps per row.
// Tables of the tensor-core interpolation kernels (umma_interp.cu) of a
// parent level: each one-dimensional step as the dense B operand of
// tcgen05.mma kind::tf32, N rows of K values, K-major with the 128-byte
// swizzle (per 32-value K-atom: 8-row groups of 1024 bytes, row r of a group
// at r * 128, its 16-byte chunk c at position c ^ r), TF32 hi part (the FP32
// value rounded to the nearest TF32, 10 mantissa bits, ties away from zero)
// then the lo part (the FP32 rest).
static float tf32_rn(float x)
{
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u = (u + 0x1000u) & 0xffffe000u;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}

// dense [rows][K] (rows <= N), appended to img at a 1024-byte boundary
static void umma_step_image(const std::vector<double> &A, int rows, UmmaStep &st, std::vector<unsigned char> &img)
{
    const int atoms = (st.K + 31) / 32;
    st.bytes = atoms * st.N * 128;
    st.off = (int)((img.size() + 1023) / 1024 * 1024);
    img.resize((size_t)st.off + 2 * (size_t)st.bytes, 0);
    st.kmask = 0;
    for (int n = 0; n < rows; ++n)
        for (int k = 0; k < st.K; ++k) {
            const double v = A[(size_t)n * st.K + k];
            if (v == 0.0) continue;
            st.kmask |= 1u << (k / 8);
            const size_t o = (size_t)(k / 32) * st.N * 128 + (n / 8) * 1024 + (n % 8) * 128 +
                             ((((k % 32) / 4) ^ (n % 8)) << 4) + (k % 4) * 4;
            const float f = (float)v, hi = tf32_rn(f), lo = f - hi;
            std::memcpy(&img[st.off + o], &hi, 4);
            std::memcpy(&img[st.off + st.bytes + o], &lo, 4);
        }
}

static int up8(int v) { return (v + 7) / 8 * 8; }
static int up4(int v) { return (v + 3) / 4 * 4; }
static int up16(int v) { return (v + 15) / 16 * 16; }

// Up: phi (B1: rows = parent phi, extended by 16 rows that repeat the first
// ones so that reflected columns never wrap; K = child phi), then theta (B2:
// rows = parent theta; K = child theta, then from kr0 on the child theta rows
// taken at phi + pi).  Down: theta (B1: rows = child theta; K = parent theta,
// then the block taken at phi + pi), then phi (B2: rows = child phi; K =
// parent phi).  A level whose steps exceed the kernels' limits (K <= 256,
// N <= 256, tensor memory <= 512 columns) gets no tables.
static cudaError_t upload_umma_tables(DevMem &M, const PlanHost &H, const Level &Lv, DevLevel<float> &D, int *err)
{
    const Level &C = H.lv[Lv.l + 1];
    const int nthp = Lv.nth, nphp = Lv.nph, nthc = C.nth, nphc = C.nph;
    auto fits = [](const UmmaStep &st) { return st.K <= 256 && st.N <= 256 && st.K > 0 && st.N > 0; };
    cudaError_t e;
    {   // up
        UmmaStep s1, s2;
        s1.K = up8(nphc);
        s1.N = up16(nphp + 16);
        s1.kr0 = s1.K;
        s2.kr0 = up4(nthc);
        s2.K = up8(s2.kr0 + nthc);
        s2.N = up16(nthp);
        const int tiles1 = (nthc + 15) / 16, tiles2 = (nphp + 15) / 16;
        const int cols = tiles1 * s1.N + s2.N + tiles2 * s2.N;
        if (fits(s1) && fits(s2) && cols <= 512) {
            std::vector<double> b1((size_t)s1.N * s1.K, 0.0), b2((size_t)s2.N * s2.K, 0.0);
            for (int n = 0; n < nphp + 16; ++n) {
                const int u = n % nphp;
                for (int f = Lv.ph_up.ptr[u]; f < Lv.ph_up.ptr[u + 1]; ++f) b1[(size_t)n * s1.K + Lv.ph_up.idx[f]] += Lv.ph_up.coef[f];
            }
            for (int t = 0; t < nthp; ++t)
                for (int f = Lv.th_up.ptr[t]; f < Lv.th_up.ptr[t + 1]; ++f)
                    b2[(size_t)t * s2.K + (Lv.th_up.refl[f] ? s2.kr0 : 0) + Lv.th_up.idx[f]] += Lv.th_up.coef[f];
            std::vector<unsigned char> img;
            umma_step_image(b1, s1.N, s1, img);
            umma_step_image(b2, s2.N, s2, img);
            const unsigned char *d;
            if ((e = M.upload(img, &d)) != cudaSuccess) return e;
            D.um_up = d;
            D.um_up_bytes = (int)img.size();
            D.um_up1 = s1;
            D.um_up2 = s2;
        }
    }
    {   // down
        UmmaStep s1, s2;
        s1.kr0 = up4(nthp);
        s1.K = up8(s1.kr0 + nthp);
        s1.N = up16(nthc);
        s2.K = up8(nphp);
        s2.N = up16(nphc);
        s2.kr0 = s2.K;
        const int tiles1 = (nphp + 15) / 16;
        const int cols = tiles1 * s1.N + s2.N;
        if (fits(s1) && fits(s2) && cols <= 512) {
            std::vector<double> b1((size_t)s1.N * s1.K, 0.0), b2((size_t)s2.N * s2.K, 0.0);
            for (int t = 0; t < nthc; ++t)
                for (int f = Lv.th_dn.ptr[t]; f < Lv.th_dn.ptr[t + 1]; ++f)
                    b1[(size_t)t * s1.K + (Lv.th_dn.refl[f] ? s1.kr0 : 0) + Lv.th_dn.idx[f]] += Lv.th_dn.coef[f];
            for (int v = 0; v < nphc; ++v)
                for (int f = Lv.ph_dn.ptr[v]; f < Lv.ph_dn.ptr[v + 1]; ++f) b2[(size_t)v * s2.K + Lv.ph_dn.idx[f]] += Lv.ph_dn.coef[f];
            std::vector<unsigned char> img;
            umma_step_image(b1, s1.N, s1, img);
            umma_step_image(b2, s2.N, s2, img);
            const unsigned char *d;
            if ((e = M.upload(img, &d)) != cudaSuccess) return e;
            D.um_dn = d;
            D.um_dn_bytes = (int)img.size();
            D.um_dn1 = s1;
            D.um_dn2 = s2;
        }
    }
    D.um_err = err;
    const char *hook = std::getenv("MLFMA_TEST_WITHHOLD_ARRIVAL");
    D.um_test = (hook && hook[0] == '1') ? 1 : 0;
    return cudaSuccess;
}

template <class R>
cudaError_t upload_tc_tables(DevMem &, const PlanHost &, const Level &, DevLevel<R> &, int *)
{
    return cudaSuccess;
}

template <>
cudaError_t upload_tc_tables<float>(DevMem &M, const PlanHost &H, const Level &Lv, DevLevel<float> &D, int *err)
{
    return upload_umma_tables(M, H, Lv, D, err);
}

template <class R>
cudaError_t upload_parent_tables(DevMem &M, const PlanHost &H, const Level &Lv, DevLevel<R> &D, int *err)
{
    cudaError_t e;
    if ((e = upload_pairs<R>(M, Lv.shift, &D.shift)) != cudaSuccess) return e;
    if ((e = upload_pairs<R>(M, Lv.shift_xy, &D.shift_xy)) != cudaSuccess) return e;
    if ((e = upload_pairs<R>(M, Lv.gam, &D.gam)) != cudaSuccess) return e;
    {
        // down-pass groups over the child level: siblings with octants o (even) and o + 1 pair up
        const Level &Cl = H.lv[Lv.l + 1];
        std::vector<int2> g;
        const int nc = Cl.nbox();
        for (int i = 0; i < nc;) {
            if (i + 1 < nc && Cl.parent[i + 1] == Cl.parent[i] && !(Cl.octant[i] & 1) && Cl.octant[i + 1] == Cl.octant[i] + 1) {
                g.push_back(make_int2(i, i + 1));
                i += 2;
            } else {
                g.push_back(make_int2(i, -1));
                i += 1;
            }
        }
        if ((e = M.upload(g, &D.dgrp)) != cudaSuccess) return e;
        D.ndgrp = (int)g.size();
    }
    auto pack = [](const Stencil &st) {
        std::vector<Tap<R>> t(st.idx.size());
        for (size_t i = 0; i < t.size(); ++i) {
            t[i].i = st.idx[i] | ((!st.refl.empty() && st.refl[i]) ? kTapRefl : 0);
            t[i].c = (R)st.coef[i];
        }
        return t;
    };
    if ((e = M.upload(pack(Lv.th_up), &D.thu)) != cudaSuccess) return e;
    D.up_order = H.order;
    if ((e = M.upload(pack(Lv.ph_up), &D.phu)) != cudaSuccess) return e;
    if ((e = M.upload(pack(Lv.th_dn), &D.thd)) != cudaSuccess) return e;
    if ((e = M.upload(pack(Lv.ph_dn), &D.phd)) != cudaSuccess) return e;
    int longest = 0;
    for (const Stencil *st : {&Lv.th_dn, &Lv.ph_dn})
        for (size_t r = 0; r + 1 < st->ptr.size(); ++r) longest = std::max(longest, st->ptr[r + 1] - st->ptr[r]);
    D.dn_taps = 0;
    for (int tm : {16, 20, 24, 32})
        if (!D.dn_taps && longest <= tm) D.dn_taps = tm;
    if (!D.dn_taps) return cudaErrorInvalidValue;   // needs interpolation order <= 12
    auto pad = [&](const Stencil &st) {
        const int rows = (int)st.ptr.size() - 1;
        std::vector<Tap<R>> t((size_t)rows * D.dn_taps, Tap<R>{0, (R)0});
        for (int r = 0; r < rows; ++r)
            for (int e2 = st.ptr[r]; e2 < st.ptr[r + 1]; ++e2) {
                Tap<R> &tp = t[(size_t)r * D.dn_taps + (e2 - st.ptr[r])];
                tp.i = st.idx[e2] | ((!st.refl.empty() && st.refl[e2]) ? kTapRefl : 0);
                tp.c = (R)st.coef[e2];
            }
        return t;
    };
    if ((e = M.upload(pad(Lv.th_dn), &D.thd_pad)) != cudaSuccess) return e;
    if ((e = M.upload(pad(Lv.ph_dn), &D.phd_pad)) != cudaSuccess) return e;
    // rows in pairs: per pair the union of both rows' taps (source index with
    // the reflection bit), one coefficient per row, zero-padded to dn2_taps
    auto pairs = [&](const Stencil &st, std::vector<std::map<int32_t, std::pair<double, double>>> &out) {
        const int rows = (int)st.ptr.size() - 1;
        out.assign((rows + 1) / 2, {});
        for (int r = 0; r < rows; ++r)
            for (int e2 = st.ptr[r]; e2 < st.ptr[r + 1]; ++e2) {
                const int32_t key = st.idx[e2] | ((!st.refl.empty() && st.refl[e2]) ? kTapRefl : 0);
                auto &cc = out[r / 2][key];
                (r % 2 ? cc.second : cc.first) += st.coef[e2];
            }
    };
    auto pack2 = [&](const std::vector<std::map<int32_t, std::pair<double, double>>> &v, int taps) {
        std::vector<Tap2<R>> t(v.size() * (size_t)taps, Tap2<R>{0, {(R)0, (R)0}});
        for (size_t b = 0; b < v.size(); ++b) {
            int f = 0;
            for (const auto &kv : v[b]) {
                Tap2<R> &tp = t[b * taps + f++];
                tp.i = kv.first;
                tp.c[0] = (R)kv.second.first;
                tp.c[1] = (R)kv.second.second;
            }
        }
        return t;
    };
    auto widest = [](const std::vector<std::map<int32_t, std::pair<double, double>>> &a,
                     const std::vector<std::map<int32_t, std::pair<double, double>>> &b) {
        size_t w = 0;
        for (const auto *v : {&a, &b})
            for (const auto &m : *v) w = std::max(w, m.size());
        return w;
    };
    std::vector<std::map<int32_t, std::pair<double, double>>> pth, pph, puth, puph;
    pairs(Lv.th_dn, pth);
    pairs(Lv.ph_dn, pph);
    const size_t wd = widest(pth, pph);
    D.dn2_taps = 0;
    for (int tm : {16, 20, 24})
        if (!D.dn2_taps && wd <= (size_t)tm) D.dn2_taps = tm;
    if (D.dn2_taps) {
        if ((e = M.upload(pack2(pth, D.dn2_taps), &D.thd2)) != cudaSuccess) return e;
        if ((e = M.upload(pack2(pph, D.dn2_taps), &D.phd2)) != cudaSuccess) return e;
    }
    pairs(Lv.th_up, puth);
    pairs(Lv.ph_up, puph);
    const size_t wu = widest(puth, puph);
    D.up2_taps = 0;
    for (int tm : {12, 16})
        if (!D.up2_taps && wu <= (size_t)tm) D.up2_taps = tm;
    if (D.up2_taps) {
        if ((e = M.upload(pack2(puth, D.up2_taps), &D.thu2)) != cudaSuccess) return e;
        if ((e = M.upload(pack2(puph, D.up2_taps), &D.phu2)) != cudaSuccess) return e;
    }
    if constexpr (sizeof(R) == 4) {
        // the four stencils on windows (FP32 windowed kernels)
        auto upload_win = [&](const WinStencil &w, WinDev &d) -> cudaError_t {
            d = WinDev();
            if (!w.groups) return cudaSuccess;
            std::vector<float4> cf((size_t)w.groups * w.tw);
            for (size_t i = 0; i < cf.size(); ++i)
                cf[i] = make_float4((float)w.coef[4 * i], (float)w.coef[4 * i + 1], (float)w.coef[4 * i + 2],
                                    (float)w.coef[4 * i + 3]);
            cudaError_t e2;
            if ((e2 = M.upload(cf, &d.coef)) != cudaSuccess) return e2;
            if ((e2 = M.upload(w.start, &d.start)) != cudaSuccess) return e2;
            d.groups = w.groups;
            d.tw = w.tw;
            return cudaSuccess;
        };
        static_assert(kWinRows == 4, "the windowed kernels take rows in groups of four");
        if ((e = upload_win(Lv.wu_th, D.wu_th)) != cudaSuccess) return e;
        if ((e = upload_win(Lv.wu_ph, D.wu_ph)) != cudaSuccess) return e;
        if ((e = upload_win(Lv.wd_ph, D.wd_ph)) != cudaSuccess) return e;
        if ((e = upload_win(Lv.wd_th, D.wd_th)) != cudaSuccess) return e;
    }
    return upload_tc_tables<R>(M, H, Lv, D, err);
}

template <class R>
cudaError_t setup_precision(mlfma_plan_t p, ProductArgs<R> &a, const double2 *near64, const double2 *V64,
                            const std::vector<const int32_t *> &dev_ints, const std::vector<const int16_t *> &dev_ty,
                            const std::vector<const int16_t *> &dev_lty)
{
    PlanHost &H = p->host;
    DevMem &M = p->mem;
    const int Bmax = p->opts.max_batch;
    cudaError_t e;
    a.n = H.N;
    a.leaf = H.leaf;
    a.levels = H.levels;
    // near values
    if (sizeof(R) == 8) {
        a.near_val = reinterpret_cast<const R *>(near64);
    } else {
        void *d;
        if ((e = M.alloc(&d, (size_t)H.nnz * 8)) != cudaSuccess) return e;
        if ((e = launch_cast_c64_to_c32(near64, static_cast<float2 *>(d), H.nnz, 0)) != cudaSuccess) return e;
        a.near_val = static_cast<const R *>(d);
    }
    if (H.leaf >= 2) {
        const int64_t nv = H.N * (int64_t)H.lv[H.leaf].K * 2;
        if (sizeof(R) == 8) {
            a.V = reinterpret_cast<const R *>(V64);
        } else {
            void *d;
            if ((e = M.alloc(&d, (size_t)nv * 8)) != cudaSuccess) return e;
            if ((e = launch_cast_c64_to_c32(V64, static_cast<float2 *>(d), nv, 0)) != cudaSuccess) return e;
            a.V = static_cast<const R *>(d);
        }
    }
    void *d;
    // status word of the tensor-core kernels' bounded waits (0 = fine)
    if ((e = M.alloc(&d, 16)) != cudaSuccess) return e;
    if ((e = cudaMemset(d, 0, 16)) != cudaSuccess) return e;
    a.um_err = static_cast<int *>(d);
    if ((e = M.alloc(&d, (size_t)H.N * Bmax * sizeof(R))) != cudaSuccess) return e;
    a.xp = static_cast<R *>(d);
    if ((e = M.alloc(&d, (size_t)H.N * Bmax * 2 * sizeof(R))) != cudaSuccess) return e;
    a.yp = static_cast<R *>(d);
    const double cfar = -H.k * H.k * H.eta / (4.0 * M_PI);
    for (int l = 2; l <= H.leaf; ++l) {
        const Level &Lv = H.lv[l];
        DevLevel<R> &D = a.lv[l];
        D.nbox = Lv.nbox();
        D.L = Lv.L; D.nth = Lv.nth; D.nph = Lv.nph; D.K = Lv.K; D.ntype = Lv.ntype;
        const int32_t *const *ip = &dev_ints[(size_t)l * kIntSlots];
        D.grp_ptr = ip[16]; D.grp_src = ip[17]; D.pchild_ptr = ip[18];
        D.grp_ty = dev_ty[l];
        D.lty_ptr = ip[19]; D.lty = ip[20]; D.grp_lty = dev_lty[l]; D.max_lty = Lv.max_lty;
        D.nparent = H.lv[l - 1].nbox();
        D.max_grp = Lv.max_grp;
        D.il_ptr = ip[0]; D.il_src = ip[1]; D.il_type = ip[2];
        D.parent = ip[3]; D.octant = ip[4]; D.child_ptr = ip[5];
        D.thu_ptr = ip[6]; D.thu_idx = ip[7]; D.thu_refl = ip[8];
        D.phu_ptr = ip[9]; D.phu_idx = ip[10];
        D.thd_ptr = ip[11]; D.thd_idx = ip[12]; D.thd_refl = ip[13];
        D.phd_ptr = ip[14]; D.phd_idx = ip[15];
        if ((e = upload_pairs<R>(M, Lv.alpha, &D.alpha)) != cudaSuccess) return e;
        if (l < H.leaf) {
            if ((e = upload_parent_tables<R>(M, H, Lv, D, a.um_err)) != cudaSuccess) return e;
        }
        std::vector<R> w(Lv.K);
        for (int q = 0; q < Lv.K; ++q)
            w[q] = (R)((l == H.leaf ? cfar : 1.0) * Lv.wt[q / Lv.nph] * 2.0 * M_PI / Lv.nph);
        if ((e = M.upload(w, &D.wq)) != cudaSuccess) return e;
        const size_t fsz = (size_t)D.nbox * 2 * Lv.K * Bmax * 2 * sizeof(R);
        if ((e = M.alloc(&d, fsz)) != cudaSuccess) return e;
        D.S = static_cast<R *>(d);
        if ((e = M.alloc(&d, fsz)) != cudaSuccess) return e;
        D.G = static_cast<R *>(d);
    }
    return cudaSuccess;
}

mlfma_status setup_device(mlfma_plan_t p)
{
    PlanHost &H = p->host;
    DevMem &M = p->mem;
    cudaError_t e;
#define CK(x, where) do { if ((e = (x)) != cudaSuccess) return cuda_fail(e, where); } while (0)
    const int nt = (int)(H.T.size() / 3);
    const double *dV;
    const int32_t *dT;
    CK(M.upload(H.V, &dV), "upload vertices");
    CK(M.upload(H.T, &dT), "upload triangles");
    void *tq, *tv, *area, *cen, *hmax;
    CK(M.alloc(&tq, sizeof(double) * 21 * nt), "alloc geometry");
    CK(M.alloc(&tv, sizeof(double) * 9 * nt), "alloc geometry");
    CK(M.alloc(&area, sizeof(double) * nt), "alloc geometry");
    CK(M.alloc(&cen, sizeof(double) * 3 * nt), "alloc geometry");
    CK(M.alloc(&hmax, sizeof(double) * nt), "alloc geometry");
    CK(launch_mesh_geometry(dV, dT, nt, (double *)tq, (double *)tv, (double *)area, (double *)cen, (double *)hmax, 0),
       "mesh geometry");
    // RWG data in leaf order
    std::vector<int32_t> rtri(2 * H.N);
    std::vector<double> rvf(6 * H.N), rlen(H.N);
    std::vector<int32_t> ubox(H.N);
    for (int64_t i = 0; i < H.N; ++i) {
        const int64_t c = H.perm[i];
        rtri[2 * i] = H.rwg.tri[2 * c];
        rtri[2 * i + 1] = H.rwg.tri[2 * c + 1];
        for (int s = 0; s < 2; ++s)
            for (int d = 0; d < 3; ++d) rvf[6 * i + 3 * s + d] = H.V[3 * H.rwg.vfree[2 * c + s] + d];
        rlen[i] = H.rwg.len[c];
        ubox[i] = H.leaf_box[c];
    }
    DevMesh dm;
    dm.nt = nt;
    dm.tq = (const double *)tq; dm.tv = (const double *)tv; dm.tvi = dT;
    dm.area = (const double *)area; dm.cen = (const double *)cen; dm.hmax = (const double *)hmax;
    dm.n = H.N;
    CK(M.upload(rtri, &dm.rtri), "upload rwg");
    CK(M.upload(rvf, &dm.rvf), "upload rwg");
    CK(M.upload(rlen, &dm.rlen), "upload rwg");
    const int32_t *d_ubox;
    CK(M.upload(ubox, &d_ubox), "upload rwg");
    const int64_t *d_perm;
    CK(M.upload(H.perm, &d_perm), "upload perm");
    DevNear nr;
    nr.nleaf = H.lv[H.leaf].nbox();
    CK(M.upload(H.box_ptr, &nr.box_ptr), "upload near");
    CK(M.upload(H.strip_off, &nr.strip_off), "upload near");
    CK(M.upload(H.col_ptr, &nr.col_ptr), "upload near");
    CK(M.upload(H.strip_col, &nr.strip_col), "upload near");
    for (int b = 0; b < nr.nleaf; ++b) nr.max_cols = std::max(nr.max_cols, H.col_ptr[b + 1] - H.col_ptr[b]);
    nr.max_rows = H.max_leaf;
    void *near64;
    CK(M.alloc(&near64, (size_t)H.nnz * 16), "alloc near field");
    CK(launch_near_fill(dm, nr, H.k, H.eta, (double2 *)near64, 0), "near fill");
    void *V64 = nullptr;
    if (H.leaf >= 2) {
        const Level &Lf = H.lv[H.leaf];
        std::vector<double> grid(9 * (size_t)Lf.K);
        for (int q = 0; q < Lf.K; ++q) {
            const int it = q / Lf.nph, ip = q % Lf.nph;
            const double ct = Lf.ct[it], st = std::sqrt(std::max(0.0, 1 - ct * ct));
            const double cp = std::cos(Lf.ph[ip]), sp = std::sin(Lf.ph[ip]);
            const double g[9] = {st * cp, st * sp, ct, ct * cp, ct * sp, -st, -sp, cp, 0.0};
            std::memcpy(&grid[9 * (size_t)q], g, sizeof(g));
        }
        const double *d_grid, *d_bc;
        CK(M.upload(grid, &d_grid), "upload grid");
        CK(M.upload(Lf.center, &d_bc), "upload centers");
        p->d_grid = d_grid;
        p->d_bc = d_bc;
        CK(M.alloc(&V64, (size_t)H.N * Lf.K * 2 * 16), "alloc patterns");
        CK(launch_leaf_patterns(dm, d_ubox, d_bc, Lf.K, d_grid, H.k, (double2 *)V64, 0), "leaf patterns");
    }
    // integer tables shared by both precisions: 16 slots per level
    std::vector<const int32_t *> ints((size_t)H.levels * kIntSlots, nullptr);
    std::vector<const int16_t *> tys((size_t)H.levels, nullptr), ltys((size_t)H.levels, nullptr);
    for (int l = 2; l <= H.leaf; ++l) {
        const Level &Lv = H.lv[l];
        const int32_t **ip = &ints[(size_t)l * kIntSlots];
        CK(M.upload(Lv.grp_ptr, &ip[16]), "upload lists");
        CK(M.upload(Lv.grp_src, &ip[17]), "upload lists");
        CK(M.upload(H.lv[l - 1].child_ptr, &ip[18]), "upload lists");
        CK(M.upload(Lv.grp_ty, &tys[l]), "upload lists");
        CK(M.upload(Lv.grp_lty, &ltys[l]), "upload lists");
        CK(M.upload(Lv.lty_ptr, &ip[19]), "upload lists");
        CK(M.upload(Lv.lty, &ip[20]), "upload lists");
        CK(M.upload(Lv.il_ptr, &ip[0]), "upload lists");
        CK(M.upload(Lv.il_src, &ip[1]), "upload lists");
        CK(M.upload(Lv.il_type, &ip[2]), "upload lists");
        CK(M.upload(Lv.parent, &ip[3]), "upload lists");
        CK(M.upload(Lv.octant, &ip[4]), "upload lists");
        if (l < H.leaf) {
            CK(M.upload(Lv.child_ptr, &ip[5]), "upload lists");
            CK(M.upload(Lv.th_up.ptr, &ip[6]), "upload stencils");
            CK(M.upload(Lv.th_up.idx, &ip[7]), "upload stencils");
            CK(M.upload(Lv.th_up.refl, &ip[8]), "upload stencils");
            CK(M.upload(Lv.ph_up.ptr, &ip[9]), "upload stencils");
            CK(M.upload(Lv.ph_up.idx, &ip[10]), "upload stencils");
            CK(M.upload(Lv.th_dn.ptr, &ip[11]), "upload stencils");
            CK(M.upload(Lv.th_dn.idx, &ip[12]), "upload stencils");
            CK(M.upload(Lv.th_dn.refl, &ip[13]), "upload stencils");
            CK(M.upload(Lv.ph_dn.ptr, &ip[14]), "upload stencils");
            CK(M.upload(Lv.ph_dn.idx, &ip[15]), "upload stencils");
        }
    }
    p->dm = dm;
    p->d_ubox = d_ubox;
    const int prec = p->opts.precisions;
    if (prec & (1 << MLFMA_FP32)) {
        p->a32.nr = nr; p->a32.ubox = d_ubox; p->a32.perm = d_perm;
        CK(setup_precision<float>(p, p->a32, (const double2 *)near64, (const double2 *)V64, ints, tys, ltys), "setup FP32");
        p->has32 = true;
    }
    if (prec & (1 << MLFMA_FP64)) {
        p->a64.nr = nr; p->a64.ubox = d_ubox; p->a64.perm = d_perm;
        CK(setup_precision<double>(p, p->a64, (const double2 *)near64, (const double2 *)V64, ints, tys, ltys), "setup FP64");
        p->has64 = true;
    }
    const size_t stage = (size_t)H.N * p->opts.max_batch * 2 * sizeof(double);
    CK(M.alloc(&p->stage_x, stage), "alloc staging");
    CK(M.alloc(&p->stage_y, stage), "alloc staging");
    if (prec & (1 << MLFMA_FP32)) CK(prime_kernels<float>(), "kernel attributes");
    if (prec & (1 << MLFMA_FP64)) CK(prime_kernels<double>(), "kernel attributes");
    CK(cudaStreamCreateWithFlags(&p->cs.main, cudaStreamNonBlocking), "create streams");
    CK(cudaStreamCreateWithFlags(&p->cs.far, cudaStreamNonBlocking), "create streams");
    CK(cudaStreamCreateWithFlags(&p->cs.tr, cudaStreamNonBlocking), "create streams");
    for (auto &ev : p->cs.ev) CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "create events");
    CK(cudaEventCreateWithFlags(&p->ev_in, cudaEventDisableTiming), "create events");
    CK(cudaEventCreateWithFlags(&p->ev_out, cudaEventDisableTiming), "create events");
    CK(cudaEventCreate(&p->clock.start), "create events");
    for (auto &ev : p->clock.ev) CK(cudaEventCreate(&ev), "create events");
    CK(cudaDeviceSynchronize(), "plan setup");
    if (!p->has64) {
        M.release(near64);
        if (V64) M.release(V64);
    }
#undef CK
    return MLFMA_OK;
}

// Tables of dZ/dk for one precision: near blocks (FP64 fill), derivative
// patterns dV/dk and dV/dk + (2/k) V, and the derivatives of the translation
// and shift tables.  Allocates; runs once per precision, outside any capture.
template <class R>
cudaError_t setup_dk(mlfma_plan_t p, ProductArgs<R> &a)
{
    PlanHost &H = p->host;
    DevMem &M = p->mem;
    cudaError_t e;
    void *near64 = nullptr, *Vd64 = nullptr, *Wd64 = nullptr;
    if ((e = M.alloc(&near64, (size_t)H.nnz * 16)) != cudaSuccess) return e;
    if ((e = launch_near_fill_dk(p->dm, a.nr, H.k, H.eta, (double2 *)near64, 0)) != cudaSuccess) return e;
    int64_t nv = 0;
    if (H.leaf >= 2) {
        const Level &Lf = H.lv[H.leaf];
        nv = H.N * (int64_t)Lf.K * 2;
        if ((e = M.alloc(&Vd64, (size_t)nv * 16)) != cudaSuccess) return e;
        if ((e = M.alloc(&Wd64, (size_t)nv * 16)) != cudaSuccess) return e;
        if ((e = launch_leaf_patterns(p->dm, p->d_ubox, p->d_bc, Lf.K, p->d_grid, H.k, (double2 *)Vd64, 0, 1)) !=
            cudaSuccess)
            return e;
        if ((e = launch_leaf_patterns(p->dm, p->d_ubox, p->d_bc, Lf.K, p->d_grid, H.k, (double2 *)Wd64, 0, 2)) !=
            cudaSuccess)
            return e;
    }
    if (sizeof(R) == 8) {
        a.near_dk = static_cast<const R *>(near64);
        a.Vd = static_cast<const R *>(Vd64);
        a.Wd = static_cast<const R *>(Wd64);
    } else {
        auto narrow = [&](void *src, int64_t n, const R **out) -> cudaError_t {
            void *d;
            cudaError_t e2 = M.alloc(&d, (size_t)n * 8);
            if (e2 != cudaSuccess) return e2;
            if ((e2 = launch_cast_c64_to_c32(static_cast<const double2 *>(src), static_cast<float2 *>(d), n, 0)) !=
                cudaSuccess)
                return e2;
            *out = static_cast<const R *>(d);
            return cudaSuccess;
        };
        if ((e = narrow(near64, H.nnz, &a.near_dk)) != cudaSuccess) return e;
        if (H.leaf >= 2) {
            if ((e = narrow(Vd64, nv, &a.Vd)) != cudaSuccess) return e;
            if ((e = narrow(Wd64, nv, &a.Wd)) != cudaSuccess) return e;
        }
    }
    for (int l = 2; l <= H.leaf; ++l) {
        const Level &Lv = H.lv[l];
        auto pairs = [](const std::vector<cd> &v) {
            std::vector<R> t(2 * v.size());
            for (size_t i = 0; i < v.size(); ++i) { t[2 * i] = (R)v[i].real(); t[2 * i + 1] = (R)v[i].imag(); }
            return t;
        };
        if ((e = M.upload(pairs(Lv.alpha_dk), &a.lv[l].alpha_dk)) != cudaSuccess) return e;
        if (l < H.leaf && (e = M.upload(pairs(Lv.shift_dk), &a.lv[l].shift_dk)) != cudaSuccess) return e;
    }
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return e;
    if (sizeof(R) == 4) {
        M.release(near64);
        if (Vd64) M.release(Vd64);
        if (Wd64) M.release(Wd64);
    }
    return cudaSuccess;
}

// FP64 near values of a strip structure, reduced to one part and stored as
// (value, 0) in precision R.
template <class R>
cudaError_t near_part(mlfma_plan_t p, const DevNear &nr, int64_t nnz, int part, const R **out)
{
    DevMem &M = p->mem;
    cudaError_t e;
    void *full, *dst;
    if ((e = M.alloc(&full, (size_t)nnz * 16)) != cudaSuccess) return e;
    if ((e = launch_near_fill(p->dm, nr, p->host.k, p->host.eta, (double2 *)full, 0)) != cudaSuccess) return e;
    if ((e = M.alloc(&dst, (size_t)nnz * 2 * sizeof(R))) != cudaSuccess) return e;
    e = sizeof(R) == 8 ? launch_part_c64((const double2 *)full, (double2 *)dst, nnz, part, 0)
                       : launch_part_c32((const double2 *)full, (float2 *)dst, nnz, part, 0);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return e;
    M.release(full);
    *out = static_cast<const R *>(dst);
    return cudaSuccess;
}

// X u (Eq. (XI)): the standard tree, near blocks Im Z, translation table
// sum i^l (2l+1) y_l P_l (Eq. (CosKer)'s alpha times -i, so that the far
// constant -k^2 eta / 4 pi of the Z product carries over).
template <class R>
cudaError_t setup_x(mlfma_plan_t p, const ProductArgs<R> &a, ProductArgs<R> &ax)
{
    const PlanHost &H = p->host;
    cudaError_t e;
    ax = a;
    if ((e = near_part<R>(p, a.nr, H.nnz, 1, &ax.near_val)) != cudaSuccess) return e;
    for (int l = 2; l <= H.leaf; ++l)
        if ((e = upload_pairs<R>(p->mem, H.lv[l].alpha_y, &ax.lv[l].alpha)) != cudaSuccess) return e;
    return cudaSuccess;
}

// R u (Eq. (RI)): near part the leaf box itself; every other pair of leaf
// boxes translated once, at the level where their ancestors are siblings
// (coarsest level 1), with sum i^l (2l+1) j_l P_l (Eq. (SinKer)'s alpha
// times i).  Levels >= 2 share the fields, grids and stencils of the
// standard tree; level 1 gets its own.
template <class R>
cudaError_t setup_r(mlfma_plan_t p, const ProductArgs<R> &a, ProductArgs<R> &ar)
{
    const PlanHost &H = p->host;
    DevMem &M = p->mem;
    const int Bmax = p->opts.max_batch;
    cudaError_t e;
    ar = a;
    DevNear sn = a.nr;
    if ((e = M.upload(H.self_off, &sn.strip_off)) != cudaSuccess) return e;
    if ((e = M.upload(H.self_col_ptr, &sn.col_ptr)) != cudaSuccess) return e;
    if ((e = M.upload(H.self_col, &sn.strip_col)) != cudaSuccess) return e;
    sn.max_cols = H.max_leaf;
    ar.nr = sn;
    if ((e = near_part<R>(p, sn, H.self_nnz, 0, &ar.near_val)) != cudaSuccess) return e;
    ar.coarsest = 1;
    for (int l = 1; l <= H.leaf; ++l) {
        const Level &Lv = H.lv[l];
        const SibLevel &S = H.sib[l];
        DevLevel<R> &D = ar.lv[l];
        if (l == 1) {
            D = DevLevel<R>();
            D.nbox = Lv.nbox();
            D.L = Lv.L; D.nth = Lv.nth; D.nph = Lv.nph; D.K = Lv.K;
            if ((e = M.upload(Lv.parent, &D.parent)) != cudaSuccess) return e;
            if ((e = M.upload(Lv.octant, &D.octant)) != cudaSuccess) return e;
            if ((e = M.upload(Lv.child_ptr, &D.child_ptr)) != cudaSuccess) return e;
            if ((e = M.upload(H.lv[0].child_ptr, &D.pchild_ptr)) != cudaSuccess) return e;
            if ((e = upload_parent_tables<R>(M, H, Lv, D, nullptr)) != cudaSuccess) return e;
            std::vector<R> w(Lv.K);
            for (int q = 0; q < Lv.K; ++q) w[q] = (R)(Lv.wt[q / Lv.nph] * 2.0 * M_PI / Lv.nph);
            if ((e = M.upload(w, &D.wq)) != cudaSuccess) return e;
            void *d;
            const size_t fsz = (size_t)D.nbox * 2 * Lv.K * Bmax * 2 * sizeof(R);
            if ((e = M.alloc(&d, fsz)) != cudaSuccess) return e;
            D.S = static_cast<R *>(d);
            if ((e = M.alloc(&d, fsz)) != cudaSuccess) return e;
            D.G = static_cast<R *>(d);
        }
        D.nparent = H.lv[l - 1].nbox();
        D.ntype = S.ntype;
        D.max_grp = S.max_grp;
        if ((e = M.upload(S.grp_ptr, &D.grp_ptr)) != cudaSuccess) return e;
        if ((e = M.upload(S.grp_src, &D.grp_src)) != cudaSuccess) return e;
        if ((e = M.upload(S.grp_ty, &D.grp_ty)) != cudaSuccess) return e;
        D.lty_ptr = nullptr; D.lty = nullptr; D.grp_lty = nullptr; D.max_lty = 0;
        D.il_ptr = nullptr; D.il_src = nullptr; D.il_type = nullptr;   // the standard lists do not apply
        if ((e = upload_pairs<R>(M, S.alpha, &D.alpha)) != cudaSuccess) return e;
    }
    return cudaDeviceSynchronize();
}

void release_streams(mlfma_plan_t p);

// Device half of a plan (tables, fields, streams) for the host tables it
// already holds; on failure everything it allocated is released.
mlfma_status attach_device(mlfma_plan_s *p)
{
    if ((p->opts.precisions & 3) == 0) return fail(MLFMA_EINVAL, "no precision requested");
    int dev = p->opts.device;
    if (dev < 0) {
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    }
    p->device = dev;
    DeviceGuard g(dev);
    mlfma_status st;
    try {
        st = setup_device(p);
    } catch (const std::bad_alloc &) {
        st = fail(MLFMA_ENOMEM, "host allocation failed during device setup");
    }
    if (st != MLFMA_OK) {
        cudaDeviceSynchronize();
        release_streams(p);
        p->mem.free_all();
        return st;
    }
    p->on_device = true;
    return MLFMA_OK;
}

// Back to a host-only plan: waits for the plan's work and frees its device
// memory, streams, events and graphs.
void detach_device(mlfma_plan_s *p)
{
    if (!p->on_device && !p->cs.main) return;
    DeviceGuard g(p->device);
    cudaDeviceSynchronize();
    release_streams(p);
    p->mem.free_all();
    p->mem.bytes = 0;
    p->cs = CoreStreams();
    p->ev_in = p->ev_out = nullptr;
    p->clock = StageClock();
    p->a32 = ProductArgs<float>(); p->ax32 = ProductArgs<float>(); p->ar32 = ProductArgs<float>();
    p->a64 = ProductArgs<double>(); p->ax64 = ProductArgs<double>(); p->ar64 = ProductArgs<double>();
    p->has32 = p->has64 = false;
    for (int i = 0; i < 2; ++i) p->dk_ready[i] = p->x_ready[i] = p->r_ready[i] = false;
    p->stage_x = p->stage_y = nullptr;
    p->on_device = false;
}

// Times every candidate of every stage (serially, CUDA events on `s`,
// after one warm-up launch) and keeps the fastest; *before / *after are the
// sums of the stages' times with the built-in choices and with the chosen
// ones.  Fields are filled by one full pass first; the contents of x do not
// change the timing.
template <class R>
cudaError_t tune_args(ProductArgs<R> a, cudaStream_t s, Tuning &best, double *before, double *after)
{
    cudaError_t e;
    a.tune = Tuning();
    best = Tuning();
    if ((e = cudaMemsetAsync(a.xp, 0, (size_t)a.n * a.B * sizeof(R), s)) != cudaSuccess) return e;
    CoreStreams serial{};
    serial.main = s;
    if ((e = launch_core<R>(a, serial, nullptr)) != cudaSuccess) return e;
    cudaEvent_t e0, e1;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    // a candidate that does not apply to this plan (its launcher refuses it,
    // or its launch is rejected) is skipped and its launch error cleared
    auto time_stage = [&](int stage, int choice) -> double {
        bool ok = launch_stage<R>(a, stage, choice, s) == cudaSuccess && cudaEventRecord(e0, s) == cudaSuccess;
        for (int r = 0; ok && r < 3; ++r) ok = launch_stage<R>(a, stage, choice, s) == cudaSuccess;
        ok = ok && cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
        float ms = 0;
        ok = ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            return -1.0;
        }
        return ms / 3.0;
    };
    double tb = 0, ta = 0;
    auto pick = [&](int stage, std::initializer_list<int> choices, int &slot) {
        const double t0 = time_stage(stage, 0);
        double tmin = t0;
        slot = 0;
        for (int c : choices) {
            const double t = time_stage(stage, c);
            if (t > 0 && t < tmin * 0.98) {   // keep the built-in choice unless clearly slower
                tmin = t;
                slot = c;
            }
        }
        tb += t0;
        ta += tmin;
    };
    pick(STAGE_NEAR, {1, 2, 3}, best.near);
    if (a.leaf >= a.coarsest) {
        pick(STAGE_RADIATE, {1, 2, 3, 4, 5}, best.radiate);
        pick(STAGE_RECEIVE, {1, 2, 3, 4, 5, 6}, best.receive);
        for (int l = a.coarsest; l <= a.leaf; ++l) {
            pick(STAGE_TRANSLATE + l, {1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11}, best.tr[l]);
            if (l < a.leaf) {
                pick(STAGE_UP + l, {1, 2, 4, 8, 16, 202, 204, 208, 216, 304, 308, 316, 404, 408, 704, 708, 716}, best.up_nb[l]);
                pick(STAGE_DOWN + l, {1, 2, 4, 8, 16, 104, 108, 204, 208, 216, 304, 308, 316, 404, 408, 504, 508, 804, 808},
                     best.down_nb[l]);
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (before) *before = tb;
    if (after) *after = ta;
    return cudaStreamSynchronize(s);   // a fault of any timed launch surfaces here
}

mlfma_status check_plan(mlfma_plan_t p)
{
    if (!p) return fail(MLFMA_EINVAL, "plan is NULL");
    return MLFMA_OK;
}

void release_streams(mlfma_plan_t p)
{
    for (auto &kv : p->graphs) cudaGraphExecDestroy(kv.second);
    p->graphs.clear();
    for (cudaStream_t st : {p->cs.main, p->cs.far, p->cs.tr})
        if (st) cudaStreamDestroy(st);
    for (auto &ev : p->cs.ev)
        if (ev) cudaEventDestroy(ev);
    for (cudaEvent_t ev : {p->ev_in, p->ev_out, p->clock.start})
        if (ev) cudaEventDestroy(ev);
    for (auto &ev : p->clock.ev)
        if (ev) cudaEventDestroy(ev);
}

// The core pass (near field and far pass) for (precision, columns), captured
// once into a CUDA graph on the plan's streams and replayed afterwards.
enum { KIND_Z = 0, KIND_DK = 1, KIND_X = 2, KIND_R = 3 };

template <class R>
mlfma_status core_graph(mlfma_plan_t p, const ProductArgs<R> &a, int prec, int kind, cudaGraphExec_t *out)
{
    const int dk = kind == KIND_DK;
    auto key = std::make_pair(prec + 4 * kind, a.B);
    auto it = p->graphs.find(key);
    if (it != p->graphs.end()) {
        *out = it->second;
        return MLFMA_OK;
    }
    cudaError_t e = cudaStreamBeginCapture(p->cs.main, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "graph capture");
    cudaError_t el = dk ? launch_core_dk<R>(a, p->cs.main, nullptr) : launch_core<R>(a, p->cs, nullptr);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(p->cs.main, &g);
    if (el != cudaSuccess || e != cudaSuccess) {
        // a failed capture leaves its error as the thread's last CUDA error:
        // clear it, so that the next launch does not report it as its own
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return el != cudaSuccess ? cuda_fail(el, "core pass launch") : cuda_fail(e, "graph capture");
    }
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
    p->graphs[key] = ex;
    *out = ex;
    return MLFMA_OK;
}

template <class R>
mlfma_status run(mlfma_plan_t p, ProductArgs<R> a, int prec, const void *xd, int xc, void *yd, int Bu, int adjoint,
                 int kind, cudaStream_t s, double *stage_ms)
{
    const int dk = kind == KIND_DK;
    if (kind == KIND_Z) {
        const int tprec = prec == MLFMA_FP64 ? MLFMA_FP64 : MLFMA_FP32;   // mixed precisions: FP32 shapes
        auto t = p->tunes.find(std::make_pair(tprec, a.B));
        if (t != p->tunes.end()) a.tune = t->second;
    }
    cudaError_t e;
    if (stage_ms) {
        StageClock &clk = p->clock;
        clk.n = 0;
        CoreStreams serial{};
        serial.main = s;
        if ((e = cudaEventRecord(clk.start, s)) != cudaSuccess) return cuda_fail(e, "stage timer");
        if ((e = launch_prepare<R>(a, xd, xc, Bu, adjoint, s)) != cudaSuccess) return cuda_fail(e, "prepare");
        clk.stage[clk.n] = STAGE_PREPARE;
        if ((e = cudaEventRecord(clk.ev[clk.n++], s)) != cudaSuccess) return cuda_fail(e, "stage timer");
        if ((e = dk ? launch_core_dk<R>(a, s, &clk) : launch_core<R>(a, serial, &clk)) != cudaSuccess)
            return cuda_fail(e, "core pass");
        if ((e = launch_finalize<R>(a, yd, xc, Bu, adjoint, s)) != cudaSuccess) return cuda_fail(e, "finalize");
        clk.stage[clk.n] = STAGE_FINALIZE;
        if ((e = cudaEventRecord(clk.ev[clk.n++], s)) != cudaSuccess) return cuda_fail(e, "stage timer");
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "stage timer");
        for (int i = 0; i < STAGE_COUNT; ++i) stage_ms[i] = 0.0;
        cudaEvent_t prev = clk.start;
        for (int i = 0; i < clk.n; ++i) {
            float ms = 0;
            if ((e = cudaEventElapsedTime(&ms, prev, clk.ev[i])) != cudaSuccess) return cuda_fail(e, "stage timer");
            stage_ms[clk.stage[i]] += ms;
            prev = clk.ev[i];
        }
        return MLFMA_OK;
    }
    if ((e = launch_prepare<R>(a, xd, xc, Bu, adjoint, s)) != cudaSuccess) return cuda_fail(e, "prepare");
    cudaGraphExec_t ex;
    mlfma_status st = core_graph<R>(p, a, prec, kind, &ex);
    if (st != MLFMA_OK) return st;
    if ((e = cudaGraphLaunch(ex, s)) != cudaSuccess) return cuda_fail(e, "graph launch");
    if ((e = launch_finalize<R>(a, yd, xc, Bu, adjoint, s)) != cudaSuccess) return cuda_fail(e, "finalize");
    return MLFMA_OK;
}

// Status word of the tensor-core kernels (after the work that may have set
// it has finished): a bounded wait that ran out is MLFMA_ETIMEOUT, once.
mlfma_status check_umma_status(mlfma_plan_t p)
{
    if (!p->has32 || !p->a32.um_err) return MLFMA_OK;
    int h = 0;
    cudaError_t e = cudaMemcpy(&h, p->a32.um_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core status");
    if (!h) return MLFMA_OK;
    if ((e = cudaMemset(p->a32.um_err, 0, sizeof(int))) != cudaSuccess) return cuda_fail(e, "tensor-core status");
    return fail(MLFMA_ETIMEOUT, "a tensor-core interpolation kernel gave up waiting for its MMAs; its output is invalid");
}

mlfma_status product(mlfma_plan_t p, const void *x, int xc, void *y, int64_t B, int prec, void *stream, int adjoint,
                     bool host, double *stage_ms = nullptr, int kind = KIND_Z)
{
    const int dk = kind == KIND_DK;
    if (check_plan(p)) return MLFMA_EINVAL;
    if (!x || !y) return fail(MLFMA_EINVAL, "x or y is NULL");
    if (B < 1) return fail(MLFMA_EINVAL, "B must be >= 1");
    // the mixed precisions are FP32 products with tensor-core interpolation
    const int key_prec = prec;
    int umma = 0;
    if (prec == MLFMA_MIXED_TF32 || prec == MLFMA_MIXED_3XTF32) {
        if (kind != KIND_Z)
            return fail(MLFMA_ENOTSUP, "the TF32 precisions apply to Z products (mlfma_matvec, _adjoint, _host)");
        umma = prec == MLFMA_MIXED_TF32 ? 1 : 3;
        prec = MLFMA_FP32;
    }
    const int64_t Bi = B * (xc ? 2 : 1);
    if (Bi > p->opts.max_batch) return fail(MLFMA_EINVAL, "B exceeds the plan's max_batch");
    {
        const int64_t rsz = prec == MLFMA_FP64 ? 8 : 4;
        if (byte_ranges_overlap(x, p->host.N * Bi * rsz, y, p->host.N * B * 2 * rsz))
            return fail(MLFMA_EINVAL, "x and y must not overlap");
    }
    if (!p->on_device) return fail(MLFMA_EINVAL, "plan was built host-only; products need a device plan");
    if (dk && 2 * Bi > p->opts.max_batch)
        return fail(MLFMA_EINVAL, "dZ/dk products carry value and tangent fields: 2 x B (x2 for complex x) must not "
                                  "exceed the plan's max_batch");
    if (prec != MLFMA_FP32 && prec != MLFMA_FP64) return fail(MLFMA_EINVAL, "unknown precision");
    if (prec == MLFMA_FP32 && !p->has32) return fail(MLFMA_EINVAL, "FP32 was not set up in this plan");
    if (prec == MLFMA_FP64 && !p->has64) return fail(MLFMA_EINVAL, "FP64 was not set up in this plan");
    DeviceGuard g(p->device);
    if (dk && !p->dk_ready[prec]) {
        cudaError_t e0 = prec == MLFMA_FP64 ? setup_dk<double>(p, p->a64) : setup_dk<float>(p, p->a32);
        if (e0 != cudaSuccess) return cuda_fail(e0, "dZ/dk tables");
        p->dk_ready[prec] = true;
    }
    if (kind == KIND_R && p->host.leaf < 2)
        return fail(MLFMA_ENOTSUP, "the sin-kernel product needs a plan with at least 3 levels");
    if (kind == KIND_X && !p->x_ready[prec]) {
        cudaError_t e0 = prec == MLFMA_FP64 ? setup_x<double>(p, p->a64, p->ax64) : setup_x<float>(p, p->a32, p->ax32);
        if (e0 != cudaSuccess) return cuda_fail(e0, "cos-kernel tables");
        p->x_ready[prec] = true;
    }
    if (kind == KIND_R && !p->r_ready[prec]) {
        cudaError_t e0 = prec == MLFMA_FP64 ? setup_r<double>(p, p->a64, p->ar64) : setup_r<float>(p, p->a32, p->ar32);
        if (e0 != cudaSuccess) return cuda_fail(e0, "sin-kernel tables");
        p->r_ready[prec] = true;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t rsz = prec == MLFMA_FP64 ? 8 : 4;
    const size_t xbytes = (size_t)p->host.N * B * (xc ? 2 : 1) * rsz;
    const size_t ybytes = (size_t)p->host.N * B * 2 * rsz;
    cudaError_t e;
    const void *xd = x;
    void *yd = y;
    if (host) {
        if ((e = cudaMemcpyAsync(p->stage_x, x, xbytes, cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return cuda_fail(e, "copy x to device");
        xd = p->stage_x;
        yd = p->stage_y;
    }
    mlfma_status st;
    if (prec == MLFMA_FP64) {
        ProductArgs<double> a = kind == KIND_X ? p->ax64 : kind == KIND_R ? p->ar64 : p->a64;
        a.B = (int)Bi;
        st = run<double>(p, a, prec, xd, xc, yd, (int)B, adjoint, kind, s, stage_ms);
    } else {
        ProductArgs<float> a = kind == KIND_X ? p->ax32 : kind == KIND_R ? p->ar32 : p->a32;
        a.B = (int)Bi;
        a.umma = umma;
        st = run<float>(p, a, key_prec, xd, xc, yd, (int)B, adjoint, kind, s, stage_ms);
    }
    if (st != MLFMA_OK) return st;
    if (host) {
        if ((e = cudaMemcpyAsync(y, p->stage_y, ybytes, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return cuda_fail(e, "copy y to host");
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "product");
        if (umma) return check_umma_status(p);
    }
    return MLFMA_OK;
}

}  // namespace

namespace mlfma {
// Read-only view of a device plan's product arguments for entry points
// defined in other translation units.  With Bi >= 1 the view carries the
// launch shapes mlfma_matvec uses for Bi internal columns (tuned or pinned,
// else built-in); Bi = 0 gives the built-in shapes.
bool plan_product_view(mlfma_plan_t p, int prec, int64_t Bi, ProductArgs<float> *a32, ProductArgs<double> *a64,
                       int *device, int *max_batch, int64_t *n)
{
    if (!p || !p->on_device) return false;
    if (prec == MLFMA_FP32 && !p->has32) return false;
    if (prec == MLFMA_FP64 && !p->has64) return false;
    if (prec == MLFMA_FP32 && a32) *a32 = p->a32;
    if (prec == MLFMA_FP64 && a64) *a64 = p->a64;
    // the launch shapes mlfma_matvec uses for these columns (tuned or pinned)
    auto t = p->tunes.find(std::make_pair(prec, (int)Bi));
    if (t != p->tunes.end()) {
        if (prec == MLFMA_FP32 && a32) a32->tune = t->second;
        if (prec == MLFMA_FP64 && a64) a64->tune = t->second;
    }
    *device = p->device;
    *max_batch = p->opts.max_batch;
    *n = p->host.N;
    return true;
}

void set_last_error(const std::string &msg) { g_err = msg; }

// Peak device bytes that mlfma_plan's device setup allocates for these host
// tables and options (every table, both FP64 setup tables, fields sized for
// max_batch, staging), used to admit plans before building them.
int64_t plan_device_bytes_estimate(const PlanHost &H, const mlfma_opts &o)
{
    const int64_t nt = (int64_t)(H.T.size() / 3), N = H.N, Bmax = o.max_batch;
    int64_t b = (int64_t)H.V.size() * 8 + (int64_t)H.T.size() * 4 + nt * (21 + 9 + 1 + 3 + 1) * 8;
    b += N * (2 * 4 + 6 * 8 + 8 + 4 + 8);
    b += (int64_t)(H.box_ptr.size() + H.col_ptr.size()) * 4 + (int64_t)H.strip_off.size() * 8 +
         (int64_t)H.strip_col.size() * 4;
    b += H.nnz * 16;
    const int64_t Kl = H.leaf >= 2 ? H.lv[H.leaf].K : 0;
    b += N * Kl * 2 * 16;
    int64_t per_prec_fields = 0, per_prec_tables = 0, ints = 0;
    for (int l = 2; l <= H.leaf; ++l) {
        const Level &Lv = H.lv[l];
        per_prec_fields += 2 * (int64_t)Lv.nbox() * 2 * Lv.K * Bmax * 2;   // S and G, complex
        per_prec_tables += (int64_t)Lv.ntype * Lv.K * 2 + 8 * (int64_t)Lv.K * 2 + Lv.K;
        ints += (int64_t)(Lv.grp_ptr.size() + Lv.grp_src.size() + Lv.il_ptr.size() + Lv.il_src.size() +
                          Lv.il_type.size() + Lv.lty_ptr.size() + Lv.lty.size() + 3 * Lv.nbox()) * 4 +
                (int64_t)(Lv.grp_ty.size() + Lv.grp_lty.size()) * 2;
    }
    b += ints;
    for (int prec = 0; prec < 2; ++prec) {
        if (!(o.precisions & (1 << prec))) continue;
        const int64_t r = prec == MLFMA_FP64 ? 8 : 4;
        if (prec == MLFMA_FP32) b += H.nnz * 8 + N * Kl * 2 * 8;
        b += N * Bmax * r * 3 + (per_prec_fields + per_prec_tables) * r;
    }
    b += 2 * N * Bmax * 2 * 8;
    return b + b / 16 + ((int64_t)64 << 20);   // allocation granularity and small tables
}

// Pieces of a Z product for callers that capture several plans into one
// graph: the core pass forked from `fork` onto the plan's streams, its
// completion recorded in the plan's own event (*done); and the input and
// output reorderings on a stream.  The plan must be a device plan with the
// precision set up; nothing here allocates.
static mlfma_status check_branch(mlfma_plan_t p, int prec, int64_t Bi)
{
    if (!p || !p->on_device) return fail(MLFMA_EINVAL, "plan is NULL or host-only");
    if (Bi < 1 || Bi > p->opts.max_batch) return fail(MLFMA_EINVAL, "columns exceed the plan's max_batch");
    if ((prec == MLFMA_FP32 && !p->has32) || (prec == MLFMA_FP64 && !p->has64) || (prec != 0 && prec != 1))
        return fail(MLFMA_EINVAL, "precision not set up in the plan");
    return MLFMA_OK;
}

mlfma_status plan_enqueue_core(mlfma_plan_t p, int prec, int64_t Bi, cudaEvent_t fork, cudaEvent_t *done)
{
    mlfma_status st = check_branch(p, prec, Bi);
    if (st != MLFMA_OK) return st;
    DeviceGuard g(p->device);
    cudaError_t e;
    if ((e = cudaStreamWaitEvent(p->cs.main, fork, 0)) != cudaSuccess) return cuda_fail(e, "fork");
    if (prec == MLFMA_FP64) {
        ProductArgs<double> a = p->a64;
        a.B = (int)Bi;
        e = launch_core<double>(a, p->cs, nullptr);
    } else {
        ProductArgs<float> a = p->a32;
        a.B = (int)Bi;
        e = launch_core<float>(a, p->cs, nullptr);
    }
    if (e != cudaSuccess) return cuda_fail(e, "core pass");
    if ((e = cudaEventRecord(p->ev_out, p->cs.main)) != cudaSuccess) return cuda_fail(e, "join");
    *done = p->ev_out;
    return MLFMA_OK;
}

mlfma_status plan_enqueue_io(mlfma_plan_t p, int prec, const void *x, int xc, void *y, int64_t B, int finalize,
                             cudaStream_t s)
{
    mlfma_status st = check_branch(p, prec, B * (xc ? 2 : 1));
    if (st != MLFMA_OK) return st;
    DeviceGuard g(p->device);
    cudaError_t e;
    if (prec == MLFMA_FP64) {
        ProductArgs<double> a = p->a64;
        a.B = (int)(B * (xc ? 2 : 1));
        e = finalize ? launch_finalize<double>(a, y, xc, (int)B, 0, s) : launch_prepare<double>(a, x, xc, (int)B, 0, s);
    } else {
        ProductArgs<float> a = p->a32;
        a.B = (int)(B * (xc ? 2 : 1));
        e = finalize ? launch_finalize<float>(a, y, xc, (int)B, 0, s) : launch_prepare<float>(a, x, xc, (int)B, 0, s);
    }
    return e == cudaSuccess ? MLFMA_OK : cuda_fail(e, finalize ? "finalize" : "prepare");
}

int64_t plan_device_bytes(mlfma_plan_t p) { return p ? p->mem.bytes : 0; }

const PlanHost *plan_host(mlfma_plan_t p) { return p ? &p->host : nullptr; }

mlfma_status plan_attach_device(mlfma_plan_t p, const mlfma_opts &o)
{
    if (!p) return fail(MLFMA_EINVAL, "plan is NULL");
    if (p->on_device) return MLFMA_OK;
    const int interp = p->opts.interp_order;
    const double eta = p->opts.eta;
    p->opts = o;
    p->opts.host_only = 0;
    p->opts.interp_order = interp;   // the host tables were built with these
    p->opts.eta = eta;
    return attach_device(p);
}

void plan_detach_device(mlfma_plan_t p)
{
    if (p) detach_device(p);
}

// Host copy of the near-field strips (leaf order, FP64 when the plan has
// FP64 values, else widened from FP32) and the plan's host tables.
bool plan_near_host(mlfma_plan_t p, std::vector<std::complex<double>> &vals, const PlanHost **host)
{
    if (!p || !p->on_device) return false;
    DeviceGuard g(p->device);
    vals.resize((size_t)p->host.nnz);
    if (p->has64) {
        if (cudaMemcpy(vals.data(), p->a64.near_val, vals.size() * 16, cudaMemcpyDeviceToHost) != cudaSuccess)
            return false;
    } else {
        std::vector<float> tmp(2 * vals.size());
        if (cudaMemcpy(tmp.data(), p->a32.near_val, tmp.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
            return false;
        for (size_t i = 0; i < vals.size(); ++i) vals[i] = std::complex<double>(tmp[2 * i], tmp[2 * i + 1]);
    }
    *host = &p->host;
    return true;
}
}  // namespace mlfma

extern "C" {

mlfma_status mlfma_default_opts(mlfma_opts *o)
{
    if (!o) return fail(MLFMA_EINVAL, "opts is NULL");
    o->interp_order = 10;
    o->max_batch = 64;
    o->precisions = (1 << MLFMA_FP32) | (1 << MLFMA_FP64);
    o->host_only = 0;
    o->device = -1;
    o->eta = 376.730313668;
    return MLFMA_OK;
}

mlfma_status mlfma_plan(const double *verts, int64_t nv, const int32_t *tris, int64_t nt, double k, int levels,
                        double digits, const mlfma_opts *opts, mlfma_plan_t *out)
{
    g_err.clear();
    if (!out) return fail(MLFMA_EINVAL, "out is NULL");
    auto t0 = std::chrono::steady_clock::now();
    std::unique_ptr<mlfma_plan_s> p(new (std::nothrow) mlfma_plan_s());
    if (!p) return fail(MLFMA_ENOMEM, "host allocation failed");
    if (opts) p->opts = *opts; else mlfma_default_opts(&p->opts);
    if (p->opts.max_batch < 1 || p->opts.max_batch > 4096) return fail(MLFMA_EINVAL, "max_batch must be in 1..4096");
    if (!(p->opts.eta > 0) || !std::isfinite(p->opts.eta)) return fail(MLFMA_EINVAL, "eta must be positive and finite");
    std::string err;
    try {
        err = build_plan_host(p->host, verts, nv, tris, nt, k, levels, digits, p->opts.interp_order, p->opts.eta);
    } catch (const std::bad_alloc &) {
        return fail(MLFMA_ENOMEM, "host allocation failed while building the plan");
    }
    if (!err.empty()) return fail(MLFMA_EINVAL, err);
    if (!p->opts.host_only) {
        mlfma_status st = attach_device(p.get());
        if (st != MLFMA_OK) return st;
    }
    p->setup_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = p.release();
    return MLFMA_OK;
}

mlfma_status mlfma_num_unknowns(mlfma_plan_t p, int64_t *n)
{
    if (check_plan(p)) return MLFMA_EINVAL;
    if (!n) return fail(MLFMA_EINVAL, "n is NULL");
    *n = p->host.N;
    return MLFMA_OK;
}

mlfma_status mlfma_rwg_edges(mlfma_plan_t p, int32_t *edge_v, int32_t *tri_pm)
{
    if (check_plan(p)) return MLFMA_EINVAL;
    if (edge_v) std::memcpy(edge_v, p->host.rwg.edge_v.data(), p->host.rwg.edge_v.size() * sizeof(int32_t));
    if (tri_pm) std::memcpy(tri_pm, p->host.rwg.tri.data(), p->host.rwg.tri.size() * sizeof(int32_t));
    return MLFMA_OK;
}

mlfma_status mlfma_matvec(mlfma_plan_t p, const void *x, int xc, void *y, int64_t B, int prec, void *stream)
{
    return product(p, x, xc, y, B, prec, stream, 0, false);
}

mlfma_status mlfma_matvec_adjoint(mlfma_plan_t p, const void *x, int xc, void *y, int64_t B, int prec, void *stream)
{
    return product(p, x, xc, y, B, prec, stream, 1, false);
}

mlfma_status mlfma_matvec_host(mlfma_plan_t p, const void *x, int xc, void *y, int64_t B, int prec, void *stream)
{
    return product(p, x, xc, y, B, prec, stream, 0, true);
}

mlfma_status mlfma_matvec_dk(mlfma_plan_t p, const void *x, int xc, void *y, int64_t B, int prec, void *stream)
{
    return product(p, x, xc, y, B, prec, stream, 0, false, nullptr, KIND_DK);
}

mlfma_status mlfma_matvec_dk_adjoint(mlfma_plan_t p, const void *x, int xc, void *y, int64_t B, int prec,
                                     void *stream)
{
    return product(p, x, xc, y, B, prec, stream, 1, false, nullptr, KIND_DK);
}

mlfma_status mlfma_tune(mlfma_plan_t p, int64_t B, int xc, int prec, void *stream, double *ms_default,
                        double *ms_tuned)
{
    if (check_plan(p)) return MLFMA_EINVAL;
    if (!p->on_device) return fail(MLFMA_EINVAL, "plan was built host-only");
    const int64_t Bi = B * (xc ? 2 : 1);
    if (B < 1 || Bi > p->opts.max_batch) return fail(MLFMA_EINVAL, "B must be in 1..max_batch");
    if ((prec == MLFMA_FP32 && !p->has32) || (prec == MLFMA_FP64 && !p->has64) || (prec != 0 && prec != 1))
        return fail(MLFMA_EINVAL, "precision not set up in this plan");
    DeviceGuard g(p->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Tuning t;
    cudaError_t e;
    if (prec == MLFMA_FP64) {
        ProductArgs<double> a = p->a64;
        a.B = (int)Bi;
        e = tune_args<double>(a, s, t, ms_default, ms_tuned);
    } else {
        ProductArgs<float> a = p->a32;
        a.B = (int)Bi;
        e = tune_args<float>(a, s, t, ms_default, ms_tuned);
    }
    if (e != cudaSuccess) return cuda_fail(e, "mlfma_tune");
    p->tunes[std::make_pair(prec, (int)Bi)] = t;
    auto it = p->graphs.find(std::make_pair(prec + 2 * KIND_Z, (int)Bi));   // recapture with the choices
    if (it != p->graphs.end()) {
        cudaGraphExecDestroy(it->second);
        p->graphs.erase(it);
    }
    return MLFMA_OK;
}

static void tuning_to_array(const Tuning &t, int32_t *c)
{
    c[0] = t.near; c[1] = t.radiate; c[2] = t.receive;
    for (int l = 0; l < MLFMA_MAX_LEVELS; ++l) {
        c[3 + l] = t.up_nb[l];
        c[3 + MLFMA_MAX_LEVELS + l] = t.down_nb[l];
        c[3 + 2 * MLFMA_MAX_LEVELS + l] = t.tr[l];
    }
}

mlfma_status mlfma_tune_get(mlfma_plan_t p, int64_t B, int xc, int prec, int32_t *choices)
{
    if (check_plan(p)) return MLFMA_EINVAL;
    if (!choices) return fail(MLFMA_EINVAL, "choices is NULL");
    auto it = p->tunes.find(std::make_pair(prec, (int)(B * (xc ? 2 : 1))));
    tuning_to_array(it == p->tunes.end() ? Tuning() : it->second, choices);
    return MLFMA_OK;
}

mlfma_status mlfma_tune_set(mlfma_plan_t p, int64_t B, int xc, int prec, const int32_t *choices)
{
    if (check_plan(p)) return MLFMA_EINVAL;
    if (!choices) return fail(MLFMA_EINVAL, "choices is NULL");
    if (B < 1 || B > p->opts.max_batch) return fail(MLFMA_EINVAL, "B must be in 1..max_batch");
    if (prec != MLFMA_FP32 && prec != MLFMA_FP64) return fail(MLFMA_EINVAL, "prec must be MLFMA_FP32 or MLFMA_FP64");
    {
        // every value must be 0 (built-in) or one of the documented shapes
        auto pow2 = [](int v) { return v == 1 || v == 2 || v == 4 || v == 8 || v == 16; };
        bool ok = choices[0] >= 0 && choices[0] <= 3 && choices[1] >= 0 && choices[1] <= 5 &&
                  choices[2] >= 0 && choices[2] <= 6;
        for (int l = 0; l < MLFMA_MAX_LEVELS && ok; ++l) {
            const int u = choices[3 + l], d = choices[3 + MLFMA_MAX_LEVELS + l], r = choices[3 + 2 * MLFMA_MAX_LEVELS + l];
            auto win = [](int x) { return x == 304 || x == 308 || x == 316 || x == 404 || x == 408; };
            ok = (u == 0 || pow2(u) || u == 202 || u == 204 || u == 208 || u == 216 || win(u) || u == 704 || u == 708 ||
                  u == 716) &&
                 (d == 0 || pow2(d) || d == 104 || d == 108 || d == 204 || d == 208 || d == 216 || win(d) || d == 504 ||
                  d == 508 || d == 804 || d == 808) &&
                 r >= 0 && r <= 11;
        }
        if (!ok) return fail(MLFMA_EINVAL, "a launch-shape choice is outside its documented set");
    }
    const int Bi = (int)(B * (xc ? 2 : 1));
    Tuning t;
    t.near = choices[0]; t.radiate = choices[1]; t.receive = choices[2];
    for (int l = 0; l < MLFMA_MAX_LEVELS; ++l) {
        t.up_nb[l] = choices[3 + l];
        t.down_nb[l] = choices[3 + MLFMA_MAX_LEVELS + l];
        t.tr[l] = choices[3 + 2 * MLFMA_MAX_LEVELS + l];
    }
    p->tunes[std::make_pair(prec, Bi)] = t;
    auto it = p->graphs.find(std::make_pair(prec + 2 * KIND_Z, Bi));
    if (it != p->graphs.end()) {
        DeviceGuard g(p->device);
        cudaDeviceSynchronize();
        cudaGraphExecDestroy(it->second);
        p->graphs.erase(it);
    }
    return MLFMA_OK;
}

mlfma_status mlfma_export_field(mlfma_plan_t p, int prec, int which, int level, int64_t B, void *dst, int64_t cap,
                                int64_t *needed)
{
    if (check_plan(p)) return MLFMA_EINVAL;
    if (!p->on_device) return fail(MLFMA_EINVAL, "plan was built host-only");
    if ((prec == MLFMA_FP32 && !p->has32) || (prec == MLFMA_FP64 && !p->has64) || (prec != 0 && prec != 1))
        return fail(MLFMA_EINVAL, "precision not set up in this plan");
    if (which != 0 && which != 1) return fail(MLFMA_EINVAL, "which must be 0 (outgoing S) or 1 (incoming G)");
    if (!(level >= 2 && level <= p->host.leaf)) return fail(MLFMA_EINVAL, "level has no far work");
    if (B < 1 || B > p->opts.max_batch) return fail(MLFMA_EINVAL, "B must be in 1..max_batch");
    const Level &Lv = p->host.lv[level];
    const size_t rsz = prec == MLFMA_FP64 ? 8 : 4;
    const size_t bytes = (size_t)Lv.nbox() * 2 * Lv.K * B * 2 * rsz;
    if (needed) *needed = (int64_t)bytes;
    if (!dst) return MLFMA_OK;
    if (cap < (int64_t)bytes) return fail(MLFMA_EINVAL, "destination too small");
    DeviceGuard g(p->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "mlfma_export_field");
    const void *src = prec == MLFMA_FP64 ? (const void *)(which ? p->a64.lv[level].G : p->a64.lv[level].S)
                                         : (const void *)(which ? p->a32.lv[level].G : p->a32.lv[level].S);
    e = cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? MLFMA_OK : cuda_fail(e, "mlfma_export_field");
}

mlfma_status mlfma_matvec_x(mlfma_plan_t p, const void *x, int xc, void *y, int64_t B, int prec, void *stream)
{
    return product(p, x, xc, y, B, prec, stream, 0, false, nullptr, KIND_X);
}

mlfma_status mlfma_matvec_r(mlfma_plan_t p, const void *x, int xc, void *y, int64_t B, int prec, void *stream)
{
    return product(p, x, xc, y, B, prec, stream, 0, false, nullptr, KIND_R);
}

mlfma_status mlfma_profile_stages(mlfma_plan_t p, const void *x, int xc, void *y, int64_t B, int prec, void *stream,
                                  double *stage_ms)
{
    if (!stage_ms) return fail(MLFMA_EINVAL, "stage_ms is NULL");
    return product(p, x, xc, y, B, prec, stream, 0, false, stage_ms);
}

mlfma_status mlfma_sync(mlfma_plan_t p, void *stream)
{
    if (check_plan(p)) return MLFMA_EINVAL;
    if (!p->on_device) return MLFMA_OK;
    DeviceGuard g(p->device);
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "mlfma_sync");
    return check_umma_status(p);
}

mlfma_status mlfma_plan_info(mlfma_plan_t p, mlfma_info *info)
{
    if (check_plan(p)) return MLFMA_EINVAL;
    if (!info) return fail(MLFMA_EINVAL, "info is NULL");
    std::memset(info, 0, sizeof(*info));
    const PlanHost &H = p->host;
    info->n = H.N;
    info->levels = H.levels;
    info->leaf_level = H.leaf;
    info->root_side = H.root_side;
    for (int d = 0; d < 3; ++d) info->root_center[d] = H.root_center[d];
    info->near_nnz = H.nnz;
    info->leaf_boxes = H.lv[H.leaf].nbox();
    info->max_leaf_unknowns = H.max_leaf;
    for (int l = 0; l < H.levels && l < MLFMA_MAX_LEVELS; ++l) {
        info->box_count[l] = H.lv[l].nbox();
        info->trunc_L[l] = H.lv[l].L;
        info->samples_K[l] = H.lv[l].K;
        info->translations[l] = (int64_t)H.lv[l].il_src.size();
    }
    info->device_bytes = p->mem.bytes;
    info->setup_seconds = p->setup_seconds;
    return MLFMA_OK;
}

mlfma_status mlfma_export(mlfma_plan_t p, int what, int level, void *dst, int64_t cap, int64_t *needed)
{
    if (check_plan(p)) return MLFMA_EINVAL;
    const PlanHost &H = p->host;
    std::vector<char> buf;
    auto put = [&](const void *src, size_t n) { buf.assign((const char *)src, (const char *)src + n); };
    const bool far_level = level >= 2 && level <= H.leaf;
    switch (what) {
    case MLFMA_X_PERM:
        put(H.perm.data(), H.perm.size() * sizeof(int64_t));
        break;
    case MLFMA_X_LEAF_BOX:
        put(H.leaf_box.data(), H.leaf_box.size() * sizeof(int32_t));
        break;
    case MLFMA_X_NEAR_COUNT:
        put(&H.nnz, sizeof(int64_t));
        break;
    case MLFMA_X_BOX_CENTERS:
        if (level < 0 || level > H.leaf) return fail(MLFMA_EINVAL, "level out of range");
        put(H.lv[level].center.data(), H.lv[level].center.size() * sizeof(double));
        break;
    case MLFMA_X_GRID: {
        if (!(far_level || (level == 1 && H.leaf >= 1))) return fail(MLFMA_EINVAL, "level has no far work");
        const Level &Lv = H.lv[level];
        std::vector<double> g(4 * (size_t)Lv.K);
        for (int q = 0; q < Lv.K; ++q) {
            g[4 * q] = Lv.ct[q / Lv.nph];
            g[4 * q + 1] = Lv.ph[q % Lv.nph];
            g[4 * q + 2] = Lv.wt[q / Lv.nph] * 2.0 * M_PI / Lv.nph;
            g[4 * q + 3] = Lv.th[q / Lv.nph];
        }
        put(g.data(), g.size() * sizeof(double));
        break;
    }
    case MLFMA_X_ALPHA:
        if (!far_level) return fail(MLFMA_EINVAL, "level has no far work");
        put(H.lv[level].alpha.data(), H.lv[level].alpha.size() * sizeof(cd));
        break;
    case MLFMA_X_ALPHA_OFFS:
        if (!far_level) return fail(MLFMA_EINVAL, "level has no far work");
        put(H.lv[level].type_off.data(), H.lv[level].type_off.size() * sizeof(int32_t));
        break;
    case MLFMA_X_ALPHA_J:
    case MLFMA_X_ALPHA_Y: {
        if (!far_level) return fail(MLFMA_EINVAL, "level has no far work");
        const std::vector<cd> &t = what == MLFMA_X_ALPHA_J ? H.lv[level].alpha_j : H.lv[level].alpha_y;
        put(t.data(), t.size() * sizeof(cd));
        break;
    }
    case MLFMA_X_SIB_ALPHA:
    case MLFMA_X_SIB_OFFS:
        if (!(level >= 1 && level <= H.leaf)) return fail(MLFMA_EINVAL, "no sibling translations at this level");
        if (what == MLFMA_X_SIB_ALPHA)
            put(H.sib[level].alpha.data(), H.sib[level].alpha.size() * sizeof(cd));
        else
            put(H.sib[level].type_off.data(), H.sib[level].type_off.size() * sizeof(int32_t));
        break;
    case MLFMA_X_SHIFT:
    case MLFMA_X_SHIFT_XY:
    case MLFMA_X_SHIFT_Z: {
        if (!(level >= 1 && level < H.leaf)) return fail(MLFMA_EINVAL, "no child-to-parent shift into this level");
        const Level &Lv = H.lv[level];
        const std::vector<cd> &t = what == MLFMA_X_SHIFT ? Lv.shift : what == MLFMA_X_SHIFT_XY ? Lv.shift_xy : Lv.gam;
        put(t.data(), t.size() * sizeof(cd));
        break;
    }
    case MLFMA_X_INTERP: {
        if (!(level >= 2 && level < H.leaf)) return fail(MLFMA_EINVAL, "no interpolation into this level");
        const Level &Pa = H.lv[level], &C = H.lv[level + 1];
        std::vector<double> Mx((size_t)Pa.K * C.K, 0.0);
        for (int t = 0; t < Pa.nth; ++t)
            for (int u = 0; u < Pa.nph; ++u)
                for (int e = Pa.ph_up.ptr[u]; e < Pa.ph_up.ptr[u + 1]; ++e) {
                    const int v0 = Pa.ph_up.idx[e];
                    for (int f = Pa.th_up.ptr[t]; f < Pa.th_up.ptr[t + 1]; ++f) {
                        const int j = Pa.th_up.idx[f];
                        const int v = Pa.th_up.refl[f] ? (v0 + C.nph / 2) % C.nph : v0;
                        Mx[(size_t)(t * Pa.nph + u) * C.K + j * C.nph + v] += Pa.ph_up.coef[e] * Pa.th_up.coef[f];
                    }
                }
        put(Mx.data(), Mx.size() * sizeof(double));
        break;
    }
    case MLFMA_X_ANTERP: {
        if (!(level >= 2 && level < H.leaf)) return fail(MLFMA_EINVAL, "no anterpolation from this level");
        const Level &Pa = H.lv[level], &C = H.lv[level + 1];
        std::vector<double> Ax((size_t)C.K * Pa.K, 0.0);
        // child (j, v') <- theta rows (t, refl) of U(t, v), U(t, v) <- phi rows u of the parent
        for (int j = 0; j < C.nth; ++j)
            for (int vp = 0; vp < C.nph; ++vp)
                for (int f = Pa.th_dn.ptr[j]; f < Pa.th_dn.ptr[j + 1]; ++f) {
                    const int t = Pa.th_dn.idx[f];
                    const int v = Pa.th_dn.refl[f] ? (vp + C.nph / 2) % C.nph : vp;
                    for (int e = Pa.ph_dn.ptr[v]; e < Pa.ph_dn.ptr[v + 1]; ++e)
                        Ax[(size_t)(j * C.nph + vp) * Pa.K + t * Pa.nph + Pa.ph_dn.idx[e]] +=
                            Pa.th_dn.coef[f] * Pa.ph_dn.coef[e];
                }
        put(Ax.data(), Ax.size() * sizeof(double));
        break;
    }
    case MLFMA_X_WIN_INTERP:
    case MLFMA_X_WIN_ANTERP: {
        if (!(level >= 2 && level < H.leaf)) return fail(MLFMA_EINVAL, "no interpolation at this level");
        const Level &Pa = H.lv[level], &C = H.lv[level + 1];
        const bool up = what == MLFMA_X_WIN_INTERP;
        const WinStencil &wt = up ? Pa.wu_th : Pa.wd_th, &wp = up ? Pa.wu_ph : Pa.wd_ph;
        if (!wt.groups || !wp.groups) return fail(MLFMA_EINVAL, "no windowed tables at this level");
        // the tables as the windowed kernels read them: theta rows r (source
        // rows n_t, columns nph_t), phi rows (source samples n_p)
        const int n_t = up ? C.nth : Pa.nth, n_p = up ? C.nph : Pa.nph;
        const int rows_t = up ? Pa.nth : C.nth, rows_p = up ? Pa.nph : C.nph;
        const int nph_t = C.nph;   // both theta steps run over the child's phi grid
        auto theta_tap = [&](int r, int f, int &src, int &refl, double &c) {
            const int g = r / kWinRows, e = wt.start[g] + f;
            c = wt.coef[((size_t)g * wt.tw + f) * kWinRows + r % kWinRows];
            refl = e < 0 || e >= n_t;
            src = e < 0 ? -e - 1 : (e >= n_t ? 2 * n_t - e - 1 : e);
        };
        auto phi_tap = [&](int r, int f, int &src, double &c) {
            const int g = r / kWinRows;
            c = wp.coef[((size_t)g * wp.tw + f) * kWinRows + r % kWinRows];
            src = (wp.start[g] + f) % n_p;
        };
        std::vector<double> M((size_t)Pa.K * C.K, 0.0);
        if (up) {
            // parent (t, u) <- phi rows u of T(t, v) <- theta rows t of the child (j, v or v + pi)
            for (int t = 0; t < rows_t; ++t)
                for (int u = 0; u < rows_p; ++u)
                    for (int e = 0; e < wp.tw; ++e) {
                        int v0;
                        double cp;
                        phi_tap(u, e, v0, cp);
                        if (cp == 0) continue;
                        for (int f = 0; f < wt.tw; ++f) {
                            int j, refl;
                            double ct;
                            theta_tap(t, f, j, refl, ct);
                            if (ct == 0) continue;
                            const int v = refl ? (v0 + nph_t / 2) % nph_t : v0;
                            M[(size_t)(t * Pa.nph + u) * C.K + j * C.nph + v] += cp * ct;
                        }
                    }
        } else {
            // child (j, v') <- theta rows j of U(t, v' or v' + pi) <- phi rows v of the parent (t, u)
            for (int j = 0; j < rows_t; ++j)
                for (int vp = 0; vp < C.nph; ++vp)
                    for (int f = 0; f < wt.tw; ++f) {
                        int t, refl;
                        double ct;
                        theta_tap(j, f, t, refl, ct);
                        if (ct == 0) continue;
                        const int v = refl ? (vp + nph_t / 2) % nph_t : vp;
                        for (int e = 0; e < wp.tw; ++e) {
                            int u;
                            double cp;
                            phi_tap(v, e, u, cp);
                            if (cp == 0) continue;
                            M[(size_t)(j * C.nph + vp) * Pa.K + t * Pa.nph + u] += ct * cp;
                        }
                    }
        }
        (void)rows_p;
        put(M.data(), M.size() * sizeof(double));
        break;
    }
    case MLFMA_X_WIN_SHAPE: {
        if (!(level >= 2 && level < H.leaf)) return fail(MLFMA_EINVAL, "no interpolation at this level");
        const Level &Pa = H.lv[level];
        int32_t sh[8];
        const WinStencil *w[4] = {&Pa.wu_th, &Pa.wu_ph, &Pa.wd_ph, &Pa.wd_th};
        for (int i = 0; i < 4; ++i) { sh[2 * i] = w[i]->groups; sh[2 * i + 1] = w[i]->tw; }
        put(sh, sizeof(sh));
        break;
    }
    default:
        return fail(MLFMA_EINVAL, "unknown table");
    }
    if (needed) *needed = (int64_t)buf.size();
    if (dst) {
        if (cap < (int64_t)buf.size()) return fail(MLFMA_EINVAL, "destination too small");
        std::memcpy(dst, buf.data(), buf.size());
    }
    return MLFMA_OK;
}

void mlfma_destroy(mlfma_plan_t p)
{
    if (!p) return;
    if (p->on_device || p->cs.main) {
        DeviceGuard g(p->device);
        cudaDeviceSynchronize();
        release_streams(p);
        p->mem.free_all();
    }
    delete p;
}

const char *mlfma_last_error(void) { return g_err.c_str(); }

}  // extern "C"
