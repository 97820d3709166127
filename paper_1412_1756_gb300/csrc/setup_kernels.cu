// FP64 setup kernels: near-field blocks of Z and leaf radiation patterns.
//
// Near field (Section III-B, first term of Eq. (ZI), Section IV "explicitly
// evaluated and stored"): Z_ij = i k eta <f_i, G, f_j> (Eq. (5)) for every
// pair of unknowns in neighbouring leaf boxes, by the seven-point degree-5
// triangle rule, with the inner 1/R and r'/R integrals in closed form for
// triangle pairs that coincide, touch, or lie closer than twice their
// longest edge (the bounded rest exp(ikR)-1)/R by the rule).  Entries whose
// triangle pairs were treated that way are averaged over both orders so
// that the stored blocks are exactly symmetric.
//
// Leaf radiation patterns (Eq. (11)): V_s,mj(khat) = int (I - khat khat) .
// f_j(r) exp(i k khat.(r_m - r)) dS, its theta and phi components.
//
// Wavenumber derivatives (quadrature, tree and samples fixed): the near
// blocks of dZ/dk = i eta (A + Phi / k^2) + i k eta (A' - Phi' / k^2), with A
// and Phi the vector- and scalar-potential parts of Z (singular parts
// extracted as above) and A', Phi' the same integrals of dg/dk = i exp(ikR)
// (bounded: plain rule); and the derivative patterns dV/dk, whose phase
// factor gains i khat.(r_m - r).
#include "device.h"

#include <algorithm>
#include <cmath>

namespace mlfma {

namespace {

__constant__ double c_rule[7][4];   // barycentric l1, l2, l3, weight (sum 1)

struct P3 {
    double x, y, z;
};
__device__ __forceinline__ P3 mk(const double *p) { return {p[0], p[1], p[2]}; }
__device__ __forceinline__ P3 operator-(P3 a, P3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ P3 operator+(P3 a, P3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ P3 operator*(double s, P3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ double dotp(P3 a, P3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ P3 crossp(P3 a, P3 b)
{
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ double lenp(P3 a) { return sqrt(dotp(a, a)); }

struct Z1 {   // complex scalar
    double re, im;
};
struct Z3 {   // complex 3-vector
    P3 re, im;
};

// ln((R+ + l+)/(R- + l-)) without cancellation: along an edge line
// (R + l)(R - l) = R0^2.
__device__ double edge_ln(double lp, double lm, double Rp, double Rm, double R0sq)
{
    if (lm >= 0.0) return log((Rp + lp) / (Rm + lm));
    if (lp <= 0.0) return log((Rm - lm) / (Rp - lp));
    return log((Rp + lp) * (Rm - lm) / R0sq);
}

// int_T dS'/R and int_T (rho' - rho)/R dS' over the flat triangle v[0..2]
// seen from r, by reduction to the three edges (in-plane divergence theorem).
__device__ void static_terms(P3 r, const P3 *v, double &J0, P3 &J1, P3 &rho)
{
    P3 nrm = crossp(v[1] - v[0], v[2] - v[0]);
    nrm = (1.0 / lenp(nrm)) * nrm;
    const double h = dotp(nrm, r - v[0]);
    const double ah = fabs(h);
    rho = r - h * nrm;
    J0 = 0.0;
    J1 = {0.0, 0.0, 0.0};
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        const P3 a = v[e], b = v[(e + 1) % 3];
        const P3 ed = b - a;
        const double el = lenp(ed);
        const P3 s = (1.0 / el) * ed;
        const P3 u = crossp(s, nrm);
        const double lp = dotp(b - rho, s), lm = dotp(a - rho, s);
        const double t = dotp(a - rho, u);
        const double R0sq = t * t + h * h;
        const double Rp = sqrt(R0sq + lp * lp), Rm = sqrt(R0sq + lm * lm);
        double f = 0.0, beta = 0.0;
        if (R0sq > 1e-28 * el * el) {
            f = edge_ln(lp, lm, Rp, Rm, R0sq);
            beta = atan2(t * lp, R0sq + ah * Rp) - atan2(t * lm, R0sq + ah * Rm);
        }
        J0 += t * f - ah * beta;
        J1 = J1 + (0.5 * (R0sq * f + lp * Rp - lm * Rm)) * u;
    }
}

// P0 = int_s g dS', P1 = int_s r' g dS' at point r.
__device__ void inner_potentials(const DevMesh &m, P3 r, int s, double k, bool singular, Z1 &P0, Z3 &P1)
{
    const double A = m.area[s];
    P0 = {0.0, 0.0};
    P1 = {{0, 0, 0}, {0, 0, 0}};
#pragma unroll
    for (int q = 0; q < 7; ++q) {
        const P3 rq = mk(m.tq + 21 * s + 3 * q);
        const double R = lenp(r - rq);
        double gr, gi;
        if (singular) {
            const double x = k * R;
            if (x < 1e-8) {
                gr = -0.5 * k * k * R;
                gi = k;
            } else {
                double sh, ch, sx, cx;
                sincos(0.5 * x, &sh, &ch);
                sincos(x, &sx, &cx);
                gr = -2.0 * sh * sh / R;
                gi = sx / R;
            }
        } else {
            double sx, cx;
            sincos(k * R, &sx, &cx);
            gr = cx / R;
            gi = sx / R;
        }
        const double w = A * c_rule[q][3];
        P0.re += w * gr;
        P0.im += w * gi;
        P1.re = P1.re + (w * gr) * rq;
        P1.im = P1.im + (w * gi) * rq;
    }
    if (singular) {
        P3 v[3] = {mk(m.tv + 9 * s), mk(m.tv + 9 * s + 3), mk(m.tv + 9 * s + 6)};
        double J0;
        P3 J1, rho;
        static_terms(r, v, J0, J1, rho);
        P0.re += J0;
        P1.re = P1.re + J1 + J0 * rho;
    }
}

__device__ bool near_singular(const DevMesh &m, int t, int s)
{
    if (t == s) return true;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            if (m.tvi[3 * t + a] == m.tvi[3 * s + b]) return true;
    const double d = lenp(mk(m.cen + 3 * t) - mk(m.cen + 3 * s));
    return d < 2.0 * fmax(m.hmax[t], m.hmax[s]);
}

// Outer triangle t of test function (sign si, length li, free vertex vi),
// inner triangle s of source function (sj, lj, vj):
// sum_p A_t w_p [ f_i(r_p) . int f_j g  -  div f_i div f_j int g / k^2 ]
template <int DSIGN = -1>
__device__ Z1 pair_integral(const DevMesh &m, int t, double si, double li, P3 vi, int s, double sj, double lj,
                            P3 vj, double k, bool singular)
{
    const double At = m.area[t], As = m.area[s];
    const double ci = si * li / (2.0 * At), cj = sj * lj / (2.0 * As);
    const double dd = (si * li / At) * (sj * lj / As) / (k * k);
    Z1 acc = {0.0, 0.0};
#pragma unroll 1
    for (int p = 0; p < 7; ++p) {
        const P3 r = mk(m.tq + 21 * t + 3 * p);
        Z1 P0;
        Z3 P1;
        inner_potentials(m, r, s, k, singular, P0, P1);
        const P3 fi = ci * (r - vi);
        // int f_j g = cj (P1 - vj P0)
        const double vre = cj * (dotp(fi, P1.re) - P0.re * dotp(fi, vj));
        const double vim = cj * (dotp(fi, P1.im) - P0.im * dotp(fi, vj));
        const double w = At * c_rule[p][3];
        if (DSIGN < 0) {
            acc.re += w * (vre - dd * P0.re);
            acc.im += w * (vim - dd * P0.im);
        } else {
            acc.re += w * (vre + dd * P0.re);
            acc.im += w * (vim + dd * P0.im);
        }
    }
    return acc;
}

// sum_p sum_q A_t w_p A_s w_q [f_i(r_p) . f_j(r_q) - div f_i div f_j / k^2] i exp(ik|r_p - r_q|)
__device__ Z1 pair_integral_dk(const DevMesh &m, int t, double si, double li, P3 vi, int s, double sj, double lj,
                               P3 vj, double k)
{
    const double At = m.area[t], As = m.area[s];
    const double ci = si * li / (2.0 * At), cj = sj * lj / (2.0 * As);
    const double dd = (si * li / At) * (sj * lj / As) / (k * k);
    Z1 acc = {0.0, 0.0};
#pragma unroll 1
    for (int p = 0; p < 7; ++p) {
        const P3 r = mk(m.tq + 21 * t + 3 * p);
        const P3 fi = ci * (r - vi);
        double are = 0.0, aim = 0.0;
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            const P3 rq = mk(m.tq + 21 * s + 3 * q);
            const double ff = dotp(fi, cj * (rq - vj)) - dd;
            double sx, cx;
            sincos(k * lenp(r - rq), &sx, &cx);
            const double w = As * c_rule[q][3] * ff;
            are -= w * sx;   // i exp(ikR) = -sin + i cos
            aim += w * cx;
        }
        const double w = At * c_rule[p][3];
        acc.re += w * are;
        acc.im += w * aim;
    }
    return acc;
}

__global__ void k_near_fill(DevMesh m, DevNear nr, double k, double eta, double2 *val)
{
    const int b = blockIdx.x;
    const int r0 = nr.box_ptr[b];
    const int nrow = nr.box_ptr[b + 1] - r0;
    const int c0 = nr.col_ptr[b];
    const int ncol = nr.col_ptr[b + 1] - c0;
    const int64_t off = nr.strip_off[b];
    const int64_t count = (int64_t)nrow * ncol;
    for (int64_t e = threadIdx.x; e < count; e += blockDim.x) {
        const int c = (int)(e / nrow), rr = (int)(e % nrow);
        const int i = r0 + rr, j = nr.strip_col[c0 + c];
        Z1 tot = {0.0, 0.0};
        for (int a = 0; a < 2; ++a) {
            const int t = m.rtri[2 * i + a];
            const double si = a == 0 ? 1.0 : -1.0;
            const P3 vi = mk(m.rvf + 6 * i + 3 * a);
            for (int bb = 0; bb < 2; ++bb) {
                const int s = m.rtri[2 * j + bb];
                const double sj = bb == 0 ? 1.0 : -1.0;
                const P3 vj = mk(m.rvf + 6 * j + 3 * bb);
                const bool sing = near_singular(m, t, s);
                Z1 z = pair_integral(m, t, si, m.rlen[i], vi, s, sj, m.rlen[j], vj, k, sing);
                if (sing) {
                    Z1 zr = pair_integral(m, s, sj, m.rlen[j], vj, t, si, m.rlen[i], vi, k, sing);
                    z.re = 0.5 * (z.re + zr.re);
                    z.im = 0.5 * (z.im + zr.im);
                }
                tot.re += z.re;
                tot.im += z.im;
            }
        }
        // multiply by i k eta
        val[off + e] = make_double2(-k * eta * tot.im, k * eta * tot.re);
    }
}

__global__ void k_near_fill_dk(DevMesh m, DevNear nr, double k, double eta, double2 *val)
{
    const int b = blockIdx.x;
    const int r0 = nr.box_ptr[b];
    const int nrow = nr.box_ptr[b + 1] - r0;
    const int c0 = nr.col_ptr[b];
    const int ncol = nr.col_ptr[b + 1] - c0;
    const int64_t off = nr.strip_off[b];
    const int64_t count = (int64_t)nrow * ncol;
    for (int64_t e = threadIdx.x; e < count; e += blockDim.x) {
        const int c = (int)(e / nrow), rr = (int)(e % nrow);
        const int i = r0 + rr, j = nr.strip_col[c0 + c];
        Z1 tv = {0.0, 0.0}, td = {0.0, 0.0};
        for (int a = 0; a < 2; ++a) {
            const int t = m.rtri[2 * i + a];
            const double si = a == 0 ? 1.0 : -1.0;
            const P3 vi = mk(m.rvf + 6 * i + 3 * a);
            for (int bb = 0; bb < 2; ++bb) {
                const int s = m.rtri[2 * j + bb];
                const double sj = bb == 0 ? 1.0 : -1.0;
                const P3 vj = mk(m.rvf + 6 * j + 3 * bb);
                const bool sing = near_singular(m, t, s);
                Z1 z = pair_integral<1>(m, t, si, m.rlen[i], vi, s, sj, m.rlen[j], vj, k, sing);
                if (sing) {
                    Z1 zr = pair_integral<1>(m, s, sj, m.rlen[j], vj, t, si, m.rlen[i], vi, k, sing);
                    z.re = 0.5 * (z.re + zr.re);
                    z.im = 0.5 * (z.im + zr.im);
                }
                tv.re += z.re;
                tv.im += z.im;
                const Z1 d = pair_integral_dk(m, t, si, m.rlen[i], vi, s, sj, m.rlen[j], vj, k);
                td.re += d.re;
                td.im += d.im;
            }
        }
        // i eta (A + Phi / k^2) + i k eta (A' - Phi' / k^2)
        val[off + e] = make_double2(-eta * tv.im - k * eta * td.im, eta * tv.re + k * eta * td.re);
    }
}

// MODE 0: V; 1: dV/dk; 2: dV/dk + (2/k) V (the receiving side's derivative
// pattern, with the k^2 of the far-field constant folded in).
template <int MODE>
__global__ void k_leaf_patterns(DevMesh m, const int32_t *ubox, const double *bc, int K, const double *grid,
                                double k, double2 *V)
{
    const int64_t total = m.n * (int64_t)K;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / K;
        const int q = (int)(idx % K);
        const P3 kh = mk(grid + 9 * q), th = mk(grid + 9 * q + 3), ph = mk(grid + 9 * q + 6);
        const P3 rc = mk(bc + 3 * ubox[i]);
        Z3 acc = {{0, 0, 0}, {0, 0, 0}};
        for (int a = 0; a < 2; ++a) {
            const int t = m.rtri[2 * i + a];
            const double sg = a == 0 ? 1.0 : -1.0;
            const P3 vf = mk(m.rvf + 6 * i + 3 * a);
            const double A = m.area[t];
            const double c = sg * m.rlen[i] / (2.0 * A);
            for (int p = 0; p < 7; ++p) {
                const P3 rp = mk(m.tq + 21 * t + 3 * p);
                const P3 f = c * (rp - vf);
                double sn, cs;
                const double ph = dotp(kh, rc - rp);
                sincos(k * ph, &sn, &cs);
                const double w = A * c_rule[p][3];
                if (MODE == 0) {
                    acc.re = acc.re + (w * cs) * f;
                    acc.im = acc.im + (w * sn) * f;
                } else {
                    // i ph exp(i k ph) (+ (2/k) exp(i k ph))
                    const double g = MODE == 2 ? 2.0 / k : 0.0;
                    acc.re = acc.re + (w * (g * cs - ph * sn)) * f;
                    acc.im = acc.im + (w * (g * sn + ph * cs)) * f;
                }
            }
        }
        V[2 * idx] = make_double2(dotp(th, acc.re), dotp(th, acc.im));
        V[2 * idx + 1] = make_double2(dotp(ph, acc.re), dotp(ph, acc.im));
    }
}

// Per-triangle geometry: quadrature points, vertices, area, centroid, longest edge.
__global__ void k_mesh_geometry(const double *V, const int32_t *T, int nt, double *tq, double *tv, double *area,
                                double *cen, double *hmax)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
        const P3 a = mk(V + 3 * T[3 * t]), b = mk(V + 3 * T[3 * t + 1]), c = mk(V + 3 * T[3 * t + 2]);
        area[t] = 0.5 * lenp(crossp(b - a, c - a));
        const P3 g = (1.0 / 3.0) * (a + b + c);
        cen[3 * t] = g.x; cen[3 * t + 1] = g.y; cen[3 * t + 2] = g.z;
        hmax[t] = fmax(lenp(b - a), fmax(lenp(c - b), lenp(a - c)));
        const P3 v[3] = {a, b, c};
        for (int i = 0; i < 3; ++i) {
            tv[9 * t + 3 * i] = v[i].x; tv[9 * t + 3 * i + 1] = v[i].y; tv[9 * t + 3 * i + 2] = v[i].z;
        }
        for (int q = 0; q < 7; ++q) {
            const P3 r = c_rule[q][0] * a + c_rule[q][1] * b + c_rule[q][2] * c;
            tq[21 * t + 3 * q] = r.x; tq[21 * t + 3 * q + 1] = r.y; tq[21 * t + 3 * q + 2] = r.z;
        }
    }
}

__global__ void k_cast(const double2 *src, float2 *dst, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double2 v = src[i];
        dst[i] = make_float2((float)v.x, (float)v.y);
    }
}

template <class C>
__global__ void k_part(const double2 *src, C *dst, int64_t n, int part)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = src[i];
        using T = decltype(C::x);
        dst[i] = C{(T)(part ? v.y : v.x), (T)0};
    }
}

cudaError_t upload_rule()
{
    // seven-point degree-5 rule (Cowper / Dunavant), weights relative to area
    const double s15 = std::sqrt(15.0);
    const double a1 = (6.0 - s15) / 21.0, a2 = (6.0 + s15) / 21.0;
    const double w1 = (155.0 - s15) / 1200.0, w2 = (155.0 + s15) / 1200.0;
    const double r[7][4] = {
        {1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0, 0.225},
        {a1, a1, 1.0 - 2.0 * a1, w1}, {a1, 1.0 - 2.0 * a1, a1, w1}, {1.0 - 2.0 * a1, a1, a1, w1},
        {a2, a2, 1.0 - 2.0 * a2, w2}, {a2, 1.0 - 2.0 * a2, a2, w2}, {1.0 - 2.0 * a2, a2, a2, w2},
    };
    return cudaMemcpyToSymbol(c_rule, r, sizeof(r));
}

}  // namespace

cudaError_t launch_mesh_geometry(const double *V, const int32_t *T, int nt, double *tq, double *tv, double *area,
                                 double *cen, double *hmax, cudaStream_t s)
{
    cudaError_t e = upload_rule();
    if (e != cudaSuccess) return e;
    int blocks = std::max(1, std::min((nt + 127) / 128, 152 * 8));
    k_mesh_geometry<<<blocks, 128, 0, s>>>(V, T, nt, tq, tv, area, cen, hmax);
    return cudaGetLastError();
}

cudaError_t launch_near_fill(const DevMesh &m, const DevNear &nr, double k, double eta, double2 *val, cudaStream_t s)
{
    cudaError_t e = upload_rule();
    if (e != cudaSuccess) return e;
    if (nr.nleaf == 0) return cudaSuccess;
    k_near_fill<<<nr.nleaf, 128, 0, s>>>(m, nr, k, eta, val);
    return cudaGetLastError();
}

cudaError_t launch_near_fill_dk(const DevMesh &m, const DevNear &nr, double k, double eta, double2 *val,
                                cudaStream_t s)
{
    cudaError_t e = upload_rule();
    if (e != cudaSuccess) return e;
    if (nr.nleaf == 0) return cudaSuccess;
    k_near_fill_dk<<<nr.nleaf, 128, 0, s>>>(m, nr, k, eta, val);
    return cudaGetLastError();
}

cudaError_t launch_leaf_patterns(const DevMesh &m, const int32_t *ubox, const double *box_center, int K,
                                 const double *grid, double k, double2 *V, cudaStream_t s, int mode)
{
    cudaError_t e = upload_rule();
    if (e != cudaSuccess) return e;
    const int64_t total = m.n * (int64_t)K;
    int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
    if (blocks < 1) blocks = 1;
    switch (mode) {
    case 0: k_leaf_patterns<0><<<blocks, 256, 0, s>>>(m, ubox, box_center, K, grid, k, V); break;
    case 1: k_leaf_patterns<1><<<blocks, 256, 0, s>>>(m, ubox, box_center, K, grid, k, V); break;
    case 2: k_leaf_patterns<2><<<blocks, 256, 0, s>>>(m, ubox, box_center, K, grid, k, V); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_part_c64(const double2 *src, double2 *dst, int64_t n, int part, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    k_part<double2><<<blocks, 256, 0, s>>>(src, dst, n, part);
    return cudaGetLastError();
}

cudaError_t launch_part_c32(const double2 *src, float2 *dst, int64_t n, int part, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    k_part<float2><<<blocks, 256, 0, s>>>(src, dst, n, part);
    return cudaGetLastError();
}

cudaError_t launch_cast_c64_to_c32(const double2 *src, float2 *dst, int64_t n, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    k_cast<<<blocks, 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

}  // namespace mlfma
