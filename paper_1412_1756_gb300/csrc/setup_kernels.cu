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

struct Z3 {   // complex 3-vector (real and imaginary parts)
    P3 re, im;
};

// ------------------------------------------------------------ near field ---
// The inner integral over a source triangle s, seen from an outer
// quadrature point r, is carried as two complex quantities:
//   psi0 = int_s g(|r - r'|) dS'          psi1 = int_s (r' - r) g(|r - r'|) dS'
// (psi1 a complex 3-vector).  For an RWG half on s with free vertex v and
// coefficient c = sign l / (2 A_s):  int f g = c (psi1 + (r - v) psi0) and
// int (div f) g = 2 c psi0.
struct SrcPot {
    double2 s;
    double2 v[3];
};

// Static (1/R) potentials of the flat triangle p[0..2] at r, written in terms
// of the distances from r to the vertices.
//
// With n the unit normal of p[0] p[1] p[2], h = n.(r - p[0]) and rho the foot
// of r in the plane, the surface gradient of R = |r - r'| with respect to r'
// is (rho' - rho) / R, and div'((rho' - rho)(R - |h|) / |rho' - rho|^2) = 1/R
// in the plane.  The divergence and gradient theorems turn both surface
// integrals into sums over the edges e = (a -> b), with outward in-plane
// normal u_e = (b - a)/|b - a| x n and d_e = (a - r).u_e:
//   int dS'/R                = sum_e d_e F_e - |h| Omega
//   int (rho' - rho)/R dS'   = sum_e u_e int_e R dl
// where F_e = int_e dl / R = ln((Ra + Rb + L) / (Ra + Rb - L)) with the
// endpoint distances Ra, Rb and the edge length L, and Omega is the solid
// angle of the triangle seen from r (van Oosterom and Strackee, IEEE TBME
// 1983: tan(Omega/2) = A.(B x C) / (Ra Rb Rc + (A.B) Rc + (B.C) Ra +
// (C.A) Rb), A, B, C the vertices relative to r).  Along the edge, with
// p = (a - r).e the position of a relative to the foot of r on the edge line
// and q the distance from r to that line,
//   int_e R dl = ((L + p) Rb - p Ra + q^2 F_e) / 2.
// (Ra + Rb)^2 - L^2 = 2 (Ra Rb + A.B) is formed without cancellation: for
// A.B < 0 as 2 |A x B|^2 / (Ra Rb - A.B).  A point on the edge segment itself
// (q = 0, where F_e diverges) contributes nothing: d_e = 0 and q = 0 there.
// Returns int dS'/R and int (r' - r)/R dS' = int (rho' - rho)/R dS' - h n int dS'/R.
__device__ void flat_static(P3 r, const P3 p[3], double &s0, P3 &s1)
{
    P3 n = crossp(p[1] - p[0], p[2] - p[0]);
    n = (1.0 / lenp(n)) * n;
    const double h = dotp(n, r - p[0]);
    const P3 A[3] = {p[0] - r, p[1] - r, p[2] - r};
    const double Rv[3] = {lenp(A[0]), lenp(A[1]), lenp(A[2])};
    double lin = 0.0;                 // sum_e d_e F_e
    P3 grad = {0.0, 0.0, 0.0};        // sum_e u_e int_e R dl
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        const int b = e == 2 ? 0 : e + 1;
        const P3 Ae = A[e], Be = A[b];
        const double Ra = Rv[e], Rb = Rv[b];
        const P3 ab = Be - Ae;
        const double L = lenp(ab);
        const P3 et = (1.0 / L) * ab;
        const P3 ue = crossp(et, n);
        const double dot = dotp(Ae, Be);
        const P3 cr = crossp(Ae, Be);
        const double cr2 = dotp(cr, cr);
        const double Q = dot >= 0.0 ? Ra * Rb + dot : cr2 / (Ra * Rb - dot);
        const double sum = Ra + Rb + L;
        const double pe = dotp(Ae, et);
        const double q2 = cr2 / (L * L);
        double Fe = 0.0;
        if (Q > 1e-30 * L * L) Fe = log(sum * sum / (2.0 * Q));
        lin += dotp(Ae, ue) * Fe;
        grad = grad + (0.5 * ((L + pe) * Rb - pe * Ra + q2 * Fe)) * ue;
    }
    const double num = dotp(A[0], crossp(A[1], A[2]));
    const double den = Rv[0] * Rv[1] * Rv[2] + dotp(A[0], A[1]) * Rv[2] + dotp(A[1], A[2]) * Rv[0] +
                       dotp(A[2], A[0]) * Rv[1];
    const double omega = fabs(2.0 * atan2(num, den));
    s0 = lin - fabs(h) * omega;
    s1 = grad - (h * s0) * n;
}

// The kernel and its smooth remainder.  exp(ikR)/R; with the static part
// taken out, (exp(ikR) - 1)/R = i k exp(ikR/2) sin(kR/2)/(kR/2), which is
// bounded (i k at R = 0) and is evaluated without a difference of close
// numbers.
__device__ __forceinline__ double2 kernel_full(double k, double R)
{
    double sn, cs;
    sincos(k * R, &sn, &cs);
    return make_double2(cs / R, sn / R);
}

__device__ __forceinline__ double2 kernel_smooth(double k, double R)
{
    const double u = 0.5 * k * R;
    double sn, cs;
    sincos(u, &sn, &cs);
    const double sc = u < 1e-4 ? 1.0 - u * u / 6.0 : sn / u;
    return make_double2(-k * sc * sn, k * sc * cs);
}

// psi0 and psi1 of source triangle s at r: seven-point rule on the kernel
// (its smooth remainder when `extract`), plus the static part in closed form.
__device__ SrcPot source_potential(const DevMesh &m, P3 r, int s, double k, bool extract)
{
    SrcPot P;
    P.s = make_double2(0.0, 0.0);
    for (int c = 0; c < 3; ++c) P.v[c] = make_double2(0.0, 0.0);
    const double As = m.area[s];
#pragma unroll
    for (int q = 0; q < 7; ++q) {
        const P3 d = mk(m.tq + 21 * s + 3 * q) - r;
        const double R = lenp(d);
        const double2 g = extract ? kernel_smooth(k, R) : kernel_full(k, R);
        const double w = As * c_rule[q][3];
        P.s.x += w * g.x;
        P.s.y += w * g.y;
        const double dc[3] = {d.x, d.y, d.z};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            P.v[c].x += w * dc[c] * g.x;
            P.v[c].y += w * dc[c] * g.y;
        }
    }
    if (extract) {
        const P3 p[3] = {mk(m.tv + 9 * s), mk(m.tv + 9 * s + 3), mk(m.tv + 9 * s + 6)};
        double s0;
        P3 s1;
        flat_static(r, p, s0, s1);
        P.s.x += s0;
        P.v[0].x += s1.x;
        P.v[1].x += s1.y;
        P.v[2].x += s1.z;
    }
    return P;
}

// Pairs whose inner integral takes the closed-form static part: the same
// triangle, triangles with a common vertex, and triangles whose centroids
// lie closer than twice the longer of their longest edges.
__device__ bool extract_pair(const DevMesh &m, int t, int s)
{
    bool touch = t == s;
    for (int x = 0; x < 9; ++x) touch = touch || m.tvi[3 * t + x / 3] == m.tvi[3 * s + x % 3];
    if (touch) return true;
    const P3 dc = mk(m.cen + 3 * t) - mk(m.cen + 3 * s);
    const double lim = 2.0 * fmax(m.hmax[t], m.hmax[s]);
    return dotp(dc, dc) < lim * lim;
}

// One RWG half on the outer triangle t (free vertex vo, coefficient co = sign
// l / (2 A_t)) against one on the inner triangle s (vi, ci): the two parts of
// Eq. (5) after integration by parts, without their constants,
//   vec = sum_p A_t w_p f_o(r_p) . int_s f_i g,   sca = sum_p A_t w_p int_s g,
// so that the pair adds i k eta (vec - 4 co ci sca / k^2) to Z.
__device__ void half_pair(const DevMesh &m, int t, double co, P3 vo, int s, double ci, P3 vi, double k,
                          bool extract, double2 &vec, double2 &sca)
{
    vec = make_double2(0.0, 0.0);
    sca = make_double2(0.0, 0.0);
    const double At = m.area[t];
#pragma unroll 1
    for (int p = 0; p < 7; ++p) {
        const P3 r = mk(m.tq + 21 * t + 3 * p);
        const SrcPot P = source_potential(m, r, s, k, extract);
        const P3 fo = co * (r - vo);
        const P3 rv = r - vi;
        // f_o . (psi1 + (r - vi) psi0) ci
        const double a0 = fo.x * ci, a1 = fo.y * ci, a2 = fo.z * ci;
        const double fr = dotp(fo, rv) * ci;
        const double w = At * c_rule[p][3];
        vec.x += w * (a0 * P.v[0].x + a1 * P.v[1].x + a2 * P.v[2].x + fr * P.s.x);
        vec.y += w * (a0 * P.v[0].y + a1 * P.v[1].y + a2 * P.v[2].y + fr * P.s.y);
        sca.x += w * P.s.x;
        sca.y += w * P.s.y;
    }
}

// The same two parts with the kernel's wavenumber derivative dg/dk =
// i exp(ikR) (bounded: seven-point rule on both triangles).
__device__ void half_pair_dk(const DevMesh &m, int t, double co, P3 vo, int s, double ci, P3 vi, double k,
                             double2 &vec, double2 &sca)
{
    vec = make_double2(0.0, 0.0);
    sca = make_double2(0.0, 0.0);
    const double At = m.area[t], As = m.area[s];
#pragma unroll 1
    for (int p = 0; p < 7; ++p) {
        const P3 r = mk(m.tq + 21 * t + 3 * p);
        const P3 fo = co * (r - vo);
        double2 pv = make_double2(0.0, 0.0), ps = make_double2(0.0, 0.0);
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            const P3 rq = mk(m.tq + 21 * s + 3 * q);
            double sn, cs;
            sincos(k * lenp(r - rq), &sn, &cs);
            const double w = As * c_rule[q][3];
            const double ff = dotp(fo, ci * (rq - vi));
            // i exp(ikR) = -sin + i cos
            pv.x -= w * ff * sn;
            pv.y += w * ff * cs;
            ps.x -= w * sn;
            ps.y += w * cs;
        }
        const double w = At * c_rule[p][3];
        vec.x += w * pv.x;
        vec.y += w * pv.y;
        sca.x += w * ps.x;
        sca.y += w * ps.y;
    }
}

// Entry (i, j) of the near field as its vector and scalar parts summed over
// the 2 x 2 triangle pairs; pairs with the static part in closed form are
// the mean of both orders (outer/inner exchanged), so the blocks are
// symmetric.  DK also returns the parts with dg/dk.
template <bool DK>
__device__ void rwg_entry(const DevMesh &m, int64_t i, int64_t j, double k, double2 &vec, double2 &sca,
                          double2 &vec_dk, double2 &sca_dk)
{
    vec = sca = vec_dk = sca_dk = make_double2(0.0, 0.0);
    for (int a = 0; a < 4; ++a) {
        const int hi = a >> 1, hj = a & 1;
        const int t = m.rtri[2 * i + hi], s = m.rtri[2 * j + hj];
        const double co = (hi ? -1.0 : 1.0) * m.rlen[i] / (2.0 * m.area[t]);
        const double ci = (hj ? -1.0 : 1.0) * m.rlen[j] / (2.0 * m.area[s]);
        const P3 vo = mk(m.rvf + 6 * i + 3 * hi), vi = mk(m.rvf + 6 * j + 3 * hj);
        const bool ex = extract_pair(m, t, s);
        double2 v1, s1;
        half_pair(m, t, co, vo, s, ci, vi, k, ex, v1, s1);
        double f = 4.0 * co * ci;
        if (ex) {
            double2 v2, s2;
            half_pair(m, s, ci, vi, t, co, vo, k, true, v2, s2);
            v1 = make_double2(0.5 * (v1.x + v2.x), 0.5 * (v1.y + v2.y));
            s1 = make_double2(0.5 * (s1.x + s2.x), 0.5 * (s1.y + s2.y));
        }
        vec.x += v1.x;
        vec.y += v1.y;
        sca.x += f * s1.x;
        sca.y += f * s1.y;
        if (DK) {
            half_pair_dk(m, t, co, vo, s, ci, vi, k, v1, s1);
            vec_dk.x += v1.x;
            vec_dk.y += v1.y;
            sca_dk.x += f * s1.x;
            sca_dk.y += f * s1.y;
        }
    }
}

// One CTA per leaf strip; threads over its (row, column) entries in the
// strip's column-major order.
//   Z      = i k eta (vec - sca / k^2)
//   dZ/dk  = i eta (vec + sca / k^2) + i k eta (vec' - sca' / k^2)
template <bool DK>
__global__ void k_near_fill(DevMesh m, DevNear nr, double k, double eta, double2 *val)
{
    const int b = blockIdx.x;
    const int r0 = nr.box_ptr[b], nrow = nr.box_ptr[b + 1] - r0;
    const int c0 = nr.col_ptr[b], ncol = nr.col_ptr[b + 1] - c0;
    const int64_t off = nr.strip_off[b];
    const int64_t count = (int64_t)nrow * ncol;
    const double ik2 = 1.0 / (k * k);
    for (int64_t e = threadIdx.x; e < count; e += blockDim.x) {
        const int64_t i = r0 + e % nrow, j = nr.strip_col[c0 + e / nrow];
        double2 vec, sca, vd, sd;
        rwg_entry<DK>(m, i, j, k, vec, sca, vd, sd);
        double2 z;
        if (!DK) {
            // i k eta (x + i y) = k eta (-y + i x)
            const double x = vec.x - ik2 * sca.x, y = vec.y - ik2 * sca.y;
            z = make_double2(-k * eta * y, k * eta * x);
        } else {
            const double x0 = vec.x + ik2 * sca.x, y0 = vec.y + ik2 * sca.y;
            const double x1 = vd.x - ik2 * sd.x, y1 = vd.y - ik2 * sd.y;
            z = make_double2(-eta * y0 - k * eta * y1, eta * x0 + k * eta * x1);
        }
        val[off + e] = z;
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
    k_near_fill<false><<<nr.nleaf, 128, 0, s>>>(m, nr, k, eta, val);
    return cudaGetLastError();
}

cudaError_t launch_near_fill_dk(const DevMesh &m, const DevNear &nr, double k, double eta, double2 *val,
                                cudaStream_t s)
{
    cudaError_t e = upload_rule();
    if (e != cudaSuccess) return e;
    if (nr.nleaf == 0) return cudaSuccess;
    k_near_fill<true><<<nr.nleaf, 128, 0, s>>>(m, nr, k, eta, val);
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
