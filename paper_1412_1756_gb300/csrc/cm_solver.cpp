// Characteristic modes by implicitly restarted Arnoldi (Section IV).
//
// Eq. (SEP1): Z^-1 R J = J / (1 + i lambda), values nearest zero = largest
// |mu|; or Eq. (SEP): X^-1 R J = J / lambda.  Each Arnoldi step applies the
// operator once: a product with R through the GPU MLFMA, then an inner
// solve (Z or X) by restarted GMRES, right-preconditioned by a sparse
// approximate inverse P of the stored near-field matrix (minimising
// ||I - Z_near P||_F over a prescribed pattern, Section IV), its products
// through the GPU MLFMA as well.  The Krylov bases, Hessenberg matrices and
// Ritz pairs are FP64 on the host; an inner solve that used FP32 products is
// checked with an FP64 product and refined when needed.
//
// Sign reading (the paper's Z = R + iX taken with exp(ikR)/R and +ik eta
// gives characteristic values of the wrong sign): with Zp the literal
// product, R := -Re Zp and X := +Im Zp, so Z_H := R + iX = -conj(Zp) and
// Z_H^-1 b = conj(Zp^-1 (-conj b)).
#include "../../include/mlfma.h"
#include "krylov.h"
#include "plan_host.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <memory>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>
#include <string>
#include <thread>
#include <vector>

namespace mlfma {
template <class R> struct ProductArgs;
bool plan_near_host(mlfma_plan_t p, std::vector<std::complex<double>> &vals, const PlanHost **host);
void set_last_error(const std::string &msg);
bool plan_product_view(mlfma_plan_t p, int prec, int64_t Bi, ProductArgs<float> *a32, ProductArgs<double> *a64, int *device,
                       int *max_batch, int64_t *n);
}  // namespace mlfma

using namespace mlfma;
using cd = std::complex<double>;

namespace {

mlfma_status fail(mlfma_status st, const std::string &msg)
{
    set_last_error(msg);
    return st;
}

double nrm2(const std::vector<cd> &v)
{
    double s = 0;
    for (const cd &z : v) s += std::norm(z);
    return std::sqrt(s);
}

cd dotc(const cd *a, const cd *b, int64_t n)   // a^H b
{
    cd s = 0;
    for (int64_t i = 0; i < n; ++i) s += std::conj(a[i]) * b[i];
    return s;
}

int host_threads() { return (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency())); }

// fn(t, i0, i1) on nt contiguous segments of [0, n), one thread each
template <class F>
void parallel_segments(int64_t n, F fn)
{
    const int nt = (int)std::max<int64_t>(1, std::min<int64_t>(host_threads(), n / 4096));
    if (nt == 1) {
        fn(0, (int64_t)0, n);
        return;
    }
    std::vector<std::thread> pool;
    for (int t = 0; t < nt; ++t)
        pool.emplace_back([&, t]() { fn(t, n * t / nt, n * (t + 1) / nt); });
    for (auto &th : pool) th.join();
}

// One classical Gram-Schmidt pass of w against V[0..k]: h_j = V_j^H w for
// all j in one sweep, then w -= sum_j h_j V_j; h is added to hcol.
void cgs_pass(const std::vector<std::vector<cd>> &V, int k, std::vector<cd> &w, cd *hcol, int64_t stride)
{
    const int64_t n = (int64_t)w.size();
    const int nt = (int)std::max<int64_t>(1, std::min<int64_t>(host_threads(), n / 4096));
    std::vector<cd> part((size_t)nt * (k + 1), 0.0);
    parallel_segments(n, [&](int t, int64_t i0, int64_t i1) {
        for (int j = 0; j <= k; ++j) part[(size_t)t * (k + 1) + j] = dotc(V[j].data() + i0, w.data() + i0, i1 - i0);
    });
    std::vector<cd> h(k + 1, 0.0);
    for (int t = 0; t < nt; ++t)
        for (int j = 0; j <= k; ++j) h[j] += part[(size_t)t * (k + 1) + j];
    parallel_segments(n, [&](int, int64_t i0, int64_t i1) {
        for (int j = 0; j <= k; ++j) {
            const cd hj = h[j];
            const cd *v = V[j].data();
            for (int64_t i = i0; i < i1; ++i) w[i] -= hj * v[i];
        }
    });
    for (int j = 0; j <= k; ++j) hcol[(int64_t)j * stride] += h[j];
}

// ------------------------------------------------- dense complex eigen ---
// Givens rotation G = [c s; -conj(s) c] (c real) with G [x; y] = [r; 0].
void givens(cd x, cd y, double &c, cd &s)
{
    const double ax = std::abs(x), ay = std::abs(y);
    if (ay == 0) { c = 1; s = 0; return; }
    if (ax == 0) { c = 0; s = std::conj(y) / ay; return; }
    const double nr = std::hypot(ax, ay);
    c = ax / nr;
    s = (x / ax) * std::conj(y) / nr;
}

// One implicitly shifted QR sweep with shift mu on rows/columns [lo, hi] of
// the m x m upper Hessenberg H (row-major); the similarity is applied to the
// whole matrix and accumulated into the columns of Q (m x m, row-major).
void qr_sweep(int m, std::vector<cd> &H, std::vector<cd> &Q, int lo, int hi, cd mu)
{
    auto h = [&](int i, int j) -> cd & { return H[(size_t)i * m + j]; };
    cd x = h(lo, lo) - mu, y = h(lo + 1, lo);
    for (int k = lo; k < hi; ++k) {
        double c;
        cd s;
        givens(x, y, c, s);
        for (int j = std::max(lo, k - 1); j < m; ++j) {   // rows k, k+1
            const cd a = h(k, j), b = h(k + 1, j);
            h(k, j) = c * a + s * b;
            h(k + 1, j) = -std::conj(s) * a + c * b;
        }
        const int rmax = std::min(k + 2, hi);
        for (int i = 0; i <= rmax; ++i) {                  // columns k, k+1
            const cd a = h(i, k), b = h(i, k + 1);
            h(i, k) = c * a + std::conj(s) * b;
            h(i, k + 1) = -s * a + c * b;
        }
        for (int i = 0; i < m; ++i) {
            cd &a = Q[(size_t)i * m + k], &b = Q[(size_t)i * m + k + 1];
            const cd qa = a, qb = b;
            a = c * qa + std::conj(s) * qb;
            b = -s * qa + c * qb;
        }
        if (k < hi - 1) {
            x = h(k + 1, k);
            y = h(k + 2, k);
        }
    }
}

// Eigenvalues w and unit eigenvectors (columns of X) of an m x m upper
// Hessenberg matrix by shifted QR (Wilkinson shifts, deflation) to Schur
// form and back-substitution.
bool hessenberg_eig(int m, std::vector<cd> H, std::vector<cd> &w, std::vector<cd> &X)
{
    std::vector<cd> Q((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i) Q[(size_t)i * m + i] = 1.0;
    auto h = [&](int i, int j) -> cd & { return H[(size_t)i * m + j]; };
    const double eps = 1e-15;
    int hi = m - 1, iter = 0, total = 0;
    while (hi > 0) {
        int l = hi;
        while (l > 0 && std::abs(h(l, l - 1)) > eps * (std::abs(h(l - 1, l - 1)) + std::abs(h(l, l)))) --l;
        if (l > 0) h(l, l - 1) = 0.0;
        if (l == hi) {
            --hi;
            iter = 0;
            continue;
        }
        const cd a = h(hi - 1, hi - 1), b = h(hi - 1, hi), c = h(hi, hi - 1), d = h(hi, hi);
        const cd tr = a + d, disc = std::sqrt(0.25 * tr * tr - (a * d - b * c));
        cd mu1 = 0.5 * tr + disc, mu2 = 0.5 * tr - disc;
        cd mu = std::abs(mu1 - d) < std::abs(mu2 - d) ? mu1 : mu2;
        if (iter > 0 && iter % 10 == 0) mu = d + cd(std::abs(c), 0.0);   // exceptional shift
        qr_sweep(m, H, Q, l, hi, mu);
        if (++iter > 60 || ++total > 100 * m) return false;
    }
    w.resize(m);
    for (int i = 0; i < m; ++i) w[i] = h(i, i);
    X.assign((size_t)m * m, 0.0);
    std::vector<cd> y(m);
    double tnorm = 0;
    for (int i = 0; i < m; ++i)
        for (int j = i; j < m; ++j) tnorm = std::max(tnorm, std::abs(h(i, j)));
    for (int j = 0; j < m; ++j) {
        std::fill(y.begin(), y.end(), 0.0);
        y[j] = 1.0;
        for (int i = j - 1; i >= 0; --i) {
            cd s = 0;
            for (int k = i + 1; k <= j; ++k) s += h(i, k) * y[k];
            cd den = h(i, i) - h(j, j);
            if (std::abs(den) < 1e-14 * tnorm) den = 1e-14 * tnorm;
            y[i] = -s / den;
        }
        double nn = 0;
        for (int i = 0; i < m; ++i) {
            cd s = 0;
            for (int k = 0; k <= j; ++k) s += Q[(size_t)i * m + k] * y[k];
            X[(size_t)i * m + j] = s;
            nn += std::norm(s);
        }
        nn = std::sqrt(nn);
        for (int i = 0; i < m; ++i) X[(size_t)i * m + j] /= nn;
    }
    return true;
}

// ---------------------------------------------- symmetric eigen (real) ---
// Eigenvalues w and orthonormal eigenvectors (columns of U, row-major m x m)
// of the symmetric m x m matrix A by cyclic Jacobi rotations (Jacobi 1846;
// the threshold-free cyclic form of Rutishauser 1966): each rotation in the
// (p, q) plane zeroes A_pq, sweeps repeat until the off-diagonal part is at
// rounding level.
void sym_eig(int m, std::vector<double> A, std::vector<double> &w, std::vector<double> &U)
{
    U.assign((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i) U[(size_t)i * m + i] = 1.0;
    auto a = [&](int i, int j) -> double & { return A[(size_t)i * m + j]; };
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0, tot = 0;
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) {
                tot += a(i, j) * a(i, j);
                if (i != j) off += a(i, j) * a(i, j);
            }
        if (off <= 1e-30 * tot) break;
        for (int pp = 0; pp < m - 1; ++pp)
            for (int q = pp + 1; q < m; ++q) {
                const double apq = a(pp, q);
                if (apq == 0) continue;
                // tan of the angle that zeroes (p, q): the smaller root of
                // t^2 + 2 theta t - 1 = 0, theta = (a_qq - a_pp) / (2 a_pq)
                const double theta = (a(q, q) - a(pp, pp)) / (2 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::abs(theta) + std::sqrt(theta * theta + 1));
                const double c = 1 / std::sqrt(t * t + 1), sn = t * c;
                for (int k = 0; k < m; ++k) {   // A J (columns p, q)
                    const double akp = a(k, pp), akq = a(k, q);
                    a(k, pp) = c * akp - sn * akq;
                    a(k, q) = sn * akp + c * akq;
                }
                for (int k = 0; k < m; ++k) {   // J^T A (rows p, q)
                    const double apk = a(pp, k), aqk = a(q, k);
                    a(pp, k) = c * apk - sn * aqk;
                    a(q, k) = sn * apk + c * aqk;
                }
                for (int k = 0; k < m; ++k) {   // U J
                    double &ukp = U[(size_t)k * m + pp], &ukq = U[(size_t)k * m + q];
                    const double x = ukp, y = ukq;
                    ukp = c * x - sn * y;
                    ukq = sn * x + c * y;
                }
            }
    }
    w.resize(m);
    for (int i = 0; i < m; ++i) w[i] = a(i, i);
}

// out (p x q, row-major) = U^T V for host blocks U [n][p], V [n][q]
void gram(int64_t n, int p, int q, const double *U, const double *V, std::vector<double> &out)
{
    const int nt = (int)std::max<int64_t>(1, std::min<int64_t>(host_threads(), n / 1024));
    std::vector<double> part((size_t)nt * p * q, 0.0);
    std::vector<std::thread> pool;
    for (int t = 0; t < nt; ++t)
        pool.emplace_back([&, t]() {
            double *acc = part.data() + (size_t)t * p * q;
            for (int64_t i = n * t / nt; i < n * (t + 1) / nt; ++i)
                for (int a = 0; a < p; ++a) {
                    const double u = U[i * p + a];
                    if (u != 0)
                        for (int b = 0; b < q; ++b) acc[(size_t)a * q + b] += u * V[i * q + b];
                }
        });
    for (auto &th : pool) th.join();
    out.assign((size_t)p * q, 0.0);
    for (int t = 0; t < nt; ++t)
        for (size_t e = 0; e < (size_t)p * q; ++e) out[e] += part[(size_t)t * p * q + e];
}

// out [n][q] = U [n][p] C (p x q, row-major)
void right_multiply(int64_t n, int p, int q, const double *U, const std::vector<double> &C, double *out)
{
    parallel_segments(n, [&](int, int64_t i0, int64_t i1) {
        for (int64_t i = i0; i < i1; ++i) {
            double *o = out + i * q;
            for (int b = 0; b < q; ++b) o[b] = 0;
            for (int a = 0; a < p; ++a) {
                const double u = U[i * p + a];
                if (u != 0)
                    for (int b = 0; b < q; ++b) o[b] += u * C[(size_t)a * q + b];
            }
        }
    });
}

// Rayleigh-Ritz for T = X^-1 R in the R inner product on span Y, from Y, R Y
// and W = T Y (so no further solve): T is self-adjoint there (R X^-1 R is
// symmetric), the projected pencil is A c = mu B c with A = (R Y)^T W and
// B = Y^T R Y (both symmetrised).  B = Ub D Ub^T; directions with D below
// 1e-9 max D carry no R energy (mu = 0 there) and are dropped; mu are the
// eigenvalues of D^-1/2 Ub^T A Ub D^-1/2 = E diag(mu) E^T (cyclic Jacobi),
// coef = Ub D^-1/2 E.  With B definite on the kept directions the Ritz
// values interlace the eigenvalues of T, so no Ritz value exceeds the
// largest |mu| = 1 / |lambda| of the pencil, whatever the inertia of X (a
// Rayleigh-Ritz step on the pencil (X, R) itself has no such bound when X is
// indefinite).  Returns the count r; mu [r] and the columns of coef [p][r]
// are sorted by |mu|, largest first.
int ritz_shift_invert(int64_t n, int p, const double *Y, const double *RY, const double *W, std::vector<double> &mu,
                      std::vector<double> &coef)
{
    std::vector<double> A, Bm;
    gram(n, p, p, RY, W, A);
    gram(n, p, p, Y, RY, Bm);
    for (int i = 0; i < p; ++i)   // symmetric parts (exactly symmetric without rounding and solve errors)
        for (int j = i + 1; j < p; ++j) {
            const double a = 0.5 * (A[(size_t)i * p + j] + A[(size_t)j * p + i]);
            const double b = 0.5 * (Bm[(size_t)i * p + j] + Bm[(size_t)j * p + i]);
            A[(size_t)i * p + j] = A[(size_t)j * p + i] = a;
            Bm[(size_t)i * p + j] = Bm[(size_t)j * p + i] = b;
        }
    std::vector<double> dv, Ub;
    sym_eig(p, Bm, dv, Ub);
    const double dmax = *std::max_element(dv.begin(), dv.end());
    std::vector<int> keep;
    for (int i = 0; i < p; ++i)
        if (dmax > 0 && dv[i] > 1e-9 * dmax) keep.push_back(i);
    const int r = (int)keep.size();
    if (r == 0) return 0;
    std::vector<double> S((size_t)p * r);   // p x r
    for (int a = 0; a < p; ++a)
        for (int j = 0; j < r; ++j) S[(size_t)a * r + j] = Ub[(size_t)a * p + keep[j]] / std::sqrt(dv[keep[j]]);
    std::vector<double> AS((size_t)p * r, 0.0), C((size_t)r * r, 0.0);
    for (int a = 0; a < p; ++a)
        for (int b = 0; b < p; ++b) {
            const double ab = A[(size_t)a * p + b];
            for (int j = 0; j < r; ++j) AS[(size_t)a * r + j] += ab * S[(size_t)b * r + j];
        }
    for (int a = 0; a < p; ++a)
        for (int i = 0; i < r; ++i)
            for (int j = 0; j < r; ++j) C[(size_t)i * r + j] += S[(size_t)a * r + i] * AS[(size_t)a * r + j];
    for (int i = 0; i < r; ++i)
        for (int j = i + 1; j < r; ++j)
            C[(size_t)i * r + j] = C[(size_t)j * r + i] = 0.5 * (C[(size_t)i * r + j] + C[(size_t)j * r + i]);
    std::vector<double> ev, E;
    sym_eig(r, C, ev, E);
    std::vector<int> order(r);
    for (int i = 0; i < r; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int x, int y) { return std::abs(ev[x]) > std::abs(ev[y]); });
    mu.resize(r);
    coef.assign((size_t)p * r, 0.0);
    for (int i = 0; i < r; ++i) {
        const int e = order[i];
        mu[i] = ev[e];
        for (int a = 0; a < p; ++a) {
            double sacc = 0;
            for (int j = 0; j < r; ++j) sacc += S[(size_t)a * r + j] * E[(size_t)j * r + e];
            coef[(size_t)a * r + i] = sacc;
        }
    }
    return r;
}

// ------------------------------------------------------- products ---
enum Which { PROD_Z, PROD_X, PROD_R };

struct Products {
    mlfma_plan_t plan;
    int64_t n;
    int prec;
    std::vector<float> xf, yf;
    std::vector<double> xd, yd;
    int64_t count = 0;

    // y = M x for complex x (host, canonical order); M = Zp, X = Im Zp or
    // R = -Re Zp (the last two through two real columns).
    mlfma_status apply(Which w, const cd *x, cd *y, int p)
    {
        const bool real_cols = w != PROD_Z;
        mlfma_status st;
        if (p == MLFMA_FP32) {
            xf.resize(2 * n);
            yf.resize(4 * n);
            for (int64_t i = 0; i < n; ++i) {
                xf[2 * i] = (float)x[i].real();
                xf[2 * i + 1] = (float)x[i].imag();
            }
            st = mlfma_matvec_host(plan, xf.data(), real_cols ? 0 : 1, yf.data(), real_cols ? 2 : 1, MLFMA_FP32, nullptr);
            if (st) return st;
            for (int64_t i = 0; i < n; ++i) {
                if (!real_cols) y[i] = cd(yf[2 * i], yf[2 * i + 1]);
                else if (w == PROD_X) y[i] = cd(yf[4 * i + 1], yf[4 * i + 3]);
                else y[i] = cd(-yf[4 * i], -yf[4 * i + 2]);
            }
        } else {
            xd.resize(2 * n);
            yd.resize(4 * n);
            for (int64_t i = 0; i < n; ++i) {
                xd[2 * i] = x[i].real();
                xd[2 * i + 1] = x[i].imag();
            }
            st = mlfma_matvec_host(plan, xd.data(), real_cols ? 0 : 1, yd.data(), real_cols ? 2 : 1, MLFMA_FP64, nullptr);
            if (st) return st;
            for (int64_t i = 0; i < n; ++i) {
                if (!real_cols) y[i] = cd(yd[2 * i], yd[2 * i + 1]);
                else if (w == PROD_X) y[i] = cd(yd[4 * i + 1], yd[4 * i + 3]);
                else y[i] = cd(-yd[4 * i], -yd[4 * i + 2]);
            }
        }
        ++count;
        return MLFMA_OK;
    }
};

// ------------------------------------------------------------ SAI ---
// P = argmin ||I - A_near P||_F over the prescribed pattern "column j of P
// lives on the unknowns of j's leaf box and its neighbours" (the near-field
// pattern; the thresholds of the paper's cited SAI variant are not given, so
// the whole near pattern is kept).  For leaf box b with unknowns J, the
// columns j in J share the support S = near unknowns of b; the rows that can
// be non-zero are those of the boxes near any box of S (the two-ring of b).
// With A = A_near[rows, S], P[S, J] solves the normal equations
// (A^H A) P = A^H E_J.  A_near is symmetric, so column s of A is row s of
// the stored strip of box(s).  P is stored in the near-strip layout (rows of
// a box x its neighbours' unknowns), so applying it is a near-field product.
struct Sai {
    const PlanHost *H = nullptr;
    std::vector<cd> vals;                 // strip layout, like the near field
    std::vector<int32_t> box_of;          // leaf-order unknown -> leaf box

    int col_offset(int a, int b) const    // first strip column of box b in box a's strip
    {
        int off = 0;
        for (int e = H->nb_ptr[a]; e < H->nb_ptr[a + 1]; ++e) {
            const int c = H->nb_box[e];
            if (c == b) return off;
            off += H->box_ptr[c + 1] - H->box_ptr[c];
        }
        return -1;
    }

    bool build(const PlanHost *host, const std::vector<cd> &near, bool imag_only)
    {
        H = host;
        const int nbox = (int)host->box_ptr.size() - 1;
        box_of.resize(host->N);
        for (int b = 0; b < nbox; ++b)
            for (int u = host->box_ptr[b]; u < host->box_ptr[b + 1]; ++u) box_of[u] = b;
        vals.assign((size_t)host->nnz, 0.0);
        const int nthreads = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
        std::vector<std::thread> pool;
        std::vector<char> bad(nthreads, 0);
        for (int t = 0; t < nthreads; ++t)
            pool.emplace_back([&, t]() {
                std::vector<int> rowpos(host->N, -1);
                for (int b = t; b < nbox; b += nthreads)
                    if (!build_box(b, near, imag_only, rowpos)) bad[t] = 1;
            });
        for (auto &th : pool) th.join();
        for (char c : bad)
            if (c) return false;
        return true;
    }

    cd z(const std::vector<cd> &near, bool imag_only, int a, int row, int col) const   // strip of a at (row, col)
    {
        const int na = H->box_ptr[a + 1] - H->box_ptr[a];
        const cd v = near[(size_t)H->strip_off[a] + (size_t)col * na + row];
        return imag_only ? cd(v.imag(), 0.0) : v;
    }

    bool build_box(int b, const std::vector<cd> &near, bool imag_only, std::vector<int> &rowpos)
    {
        const int r0 = H->box_ptr[b], nJ = H->box_ptr[b + 1] - r0;
        // support S: the strip columns of b (unknowns of b's neighbours)
        const int c0 = H->col_ptr[b], nS = H->col_ptr[b + 1] - c0;
        const int32_t *S = H->strip_col.data() + c0;
        // rows: the two-ring of b, grouped by box
        std::vector<int> ring;
        for (int e = H->nb_ptr[b]; e < H->nb_ptr[b + 1]; ++e) {
            const int a = H->nb_box[e];
            for (int f = H->nb_ptr[a]; f < H->nb_ptr[a + 1]; ++f) ring.push_back(H->nb_box[f]);
        }
        std::sort(ring.begin(), ring.end());
        ring.erase(std::unique(ring.begin(), ring.end()), ring.end());
        int nR = 0;
        std::vector<int> ring_off(ring.size() + 1);
        for (size_t i = 0; i < ring.size(); ++i) {
            ring_off[i] = nR;
            for (int u = H->box_ptr[ring[i]]; u < H->box_ptr[ring[i] + 1]; ++u) rowpos[u] = nR++;
        }
        ring_off[ring.size()] = nR;
        // A [nR x nS], column-major: column s = row s of box(s)'s strip
        std::vector<cd> A((size_t)nR * nS, 0.0);
        for (int k = 0; k < nS; ++k) {
            const int s = S[k], a = box_of[s];
            const int na = H->box_ptr[a + 1] - H->box_ptr[a];
            const int ac0 = H->col_ptr[a], anc = H->col_ptr[a + 1] - ac0;
            (void)na;
            for (int c = 0; c < anc; ++c) {
                const int r = rowpos[H->strip_col[ac0 + c]];
                A[(size_t)k * nR + r] = z(near, imag_only, a, s - H->box_ptr[a], c);
            }
        }
        // N = A^H A (Hermitian; upper triangle then mirrored)
        std::vector<cd> N((size_t)nS * nS, 0.0);
        for (int i = 0; i < nS; ++i) {
            const cd *ai = A.data() + (size_t)i * nR;
            for (int j = i; j < nS; ++j) {
                const cd *aj = A.data() + (size_t)j * nR;
                cd s = 0;
                for (int r = 0; r < nR; ++r) s += std::conj(ai[r]) * aj[r];
                N[(size_t)i * nS + j] = s;
                N[(size_t)j * nS + i] = std::conj(s);
            }
        }
        // rhs = A^H E_J: rhs[i][jj] = conj(A[row(J_jj), i])
        std::vector<cd> P((size_t)nS * nJ);
        for (int i = 0; i < nS; ++i)
            for (int jj = 0; jj < nJ; ++jj) P[(size_t)i * nJ + jj] = std::conj(A[(size_t)i * nR + rowpos[r0 + jj]]);
        for (int u : ring)
            for (int w = H->box_ptr[u]; w < H->box_ptr[u + 1]; ++w) rowpos[w] = -1;
        // Cholesky N = L L^H in place (lower), then L L^H P = rhs
        for (int j = 0; j < nS; ++j) {
            double d = N[(size_t)j * nS + j].real();
            for (int k = 0; k < j; ++k) d -= std::norm(N[(size_t)j * nS + k]);
            if (!(d > 0)) return false;
            const double ljj = std::sqrt(d);
            N[(size_t)j * nS + j] = ljj;
            for (int i = j + 1; i < nS; ++i) {
                cd s = N[(size_t)i * nS + j];
                for (int k = 0; k < j; ++k) s -= N[(size_t)i * nS + k] * std::conj(N[(size_t)j * nS + k]);
                N[(size_t)i * nS + j] = s / ljj;
            }
        }
        for (int jj = 0; jj < nJ; ++jj) {
            for (int i = 0; i < nS; ++i) {
                cd s = P[(size_t)i * nJ + jj];
                for (int k = 0; k < i; ++k) s -= N[(size_t)i * nS + k] * P[(size_t)k * nJ + jj];
                P[(size_t)i * nJ + jj] = s / N[(size_t)i * nS + i];
            }
            for (int i = nS - 1; i >= 0; --i) {
                cd s = P[(size_t)i * nJ + jj];
                for (int k = i + 1; k < nS; ++k) s -= std::conj(N[(size_t)k * nS + i]) * P[(size_t)k * nJ + jj];
                P[(size_t)i * nJ + jj] = s / N[(size_t)i * nS + i];
            }
        }
        // scatter P[S, J] into the strips of the boxes holding S
        for (int k = 0; k < nS; ++k) {
            const int s = S[k], a = box_of[s];
            const int na = H->box_ptr[a + 1] - H->box_ptr[a];
            const int off = col_offset(a, b);
            if (off < 0) return false;
            cd *strip = vals.data() + H->strip_off[a];
            for (int jj = 0; jj < nJ; ++jj) strip[(size_t)(off + jj) * na + (s - H->box_ptr[a])] = P[(size_t)k * nJ + jj];
        }
        return true;
    }

    // y = P x, canonical order in and out (near-field-shaped product)
    void apply(const cd *x, cd *y) const
    {
        const int nbox = (int)H->box_ptr.size() - 1;
        const int nthreads = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
        std::vector<std::thread> pool;
        for (int t = 0; t < nthreads; ++t)
            pool.emplace_back([&, t]() {
                for (int a = t; a < nbox; a += nthreads) {
                    const int r0 = H->box_ptr[a], na = H->box_ptr[a + 1] - r0;
                    const int c0 = H->col_ptr[a], nc = H->col_ptr[a + 1] - c0;
                    const cd *strip = vals.data() + H->strip_off[a];
                    std::vector<cd> acc(na, 0.0);
                    for (int c = 0; c < nc; ++c) {          // column-major strip: contiguous reads
                        const cd xv = x[H->perm[H->strip_col[c0 + c]]];
                        const cd *col = strip + (size_t)c * na;
                        for (int i = 0; i < na; ++i) acc[i] += col[i] * xv;
                    }
                    for (int i = 0; i < na; ++i) y[H->perm[r0 + i]] = acc[i];
                }
            });
        for (auto &th : pool) th.join();
    }
};

// --------------------------------------------------------- GMRES ---
// Solve M w = b (M = Zp or X) with right preconditioning by P, restarted
// every m iterations; FP64 Krylov arithmetic, products in precision `prec`;
// the final residual is re-checked with an FP64 product when the plan has
// one, and the solve continues from there if it is above tol.
struct Gmres {
    Products *prod;
    const Sai *sai;
    Which which;
    int prec, restart, maxit, check_prec;
    double tol;
    DeviceGmres *dev = nullptr;   // FP32 passes on the device when set
    int64_t iterations = 0;

    mlfma_status solve(const std::vector<cd> &b, std::vector<cd> &w, bool &converged)
    {
        const int64_t n = (int64_t)b.size();
        w.assign(n, 0.0);
        const double bn = nrm2(b);
        converged = false;
        if (bn == 0) {
            converged = true;
            return MLFMA_OK;
        }
        std::vector<cd> r = b, t(n), z(n);
        std::vector<std::vector<cd>> V;
        int used = 0;
        for (int refine = 0; refine < 8 && used < maxit; ++refine) {
            // inner restarted GMRES on M d = r (r = current residual)
            std::vector<cd> d(n, 0.0), rr = r;
            double rn = nrm2(rr);
            // a pass with FP32 products can lower its own residual by ~1e-5 at
            // most; the FP64 check and further passes do the rest
            const double target = std::max(0.5 * tol * bn, (prec == MLFMA_FP32 ? 1e-5 : 0.0) * rn);
            if (dev && prec == MLFMA_FP32 && rn > target) {
                std::string err;
                const int it = device_gmres_run(dev, which == PROD_Z ? 0 : 1, r.data(), d.data(), target, maxit - used,
                                                err);
                if (it < 0) return fail(MLFMA_ECUDA, err);
                used += it;
                iterations += it;
                prod->count += it;
                rn = 0.0;   // the loop below is the host path
            }
            while (used < maxit && rn > target) {
                const int m = std::min(restart, maxit - used);
                V.assign(m + 1, std::vector<cd>(n));
                std::vector<cd> Hm((size_t)(m + 1) * m, 0.0), g(m + 1, 0.0), cs(m), sn(m);
                std::vector<double> cr(m);
                for (int64_t i = 0; i < n; ++i) V[0][i] = rr[i] / rn;
                g[0] = rn;
                int k = 0;
                for (; k < m; ++k) {
                    if (sai) sai->apply(V[k].data(), z.data());
                    else z = V[k];
                    mlfma_status st = prod->apply(which, z.data(), V[k + 1].data(), prec);
                    if (st) return st;
                    ++used;
                    ++iterations;
                    for (int pass = 0; pass < 2; ++pass)   // classical Gram-Schmidt, twice
                        cgs_pass(V, k, V[k + 1], &Hm[k], m);
                    const double hn = nrm2(V[k + 1]);
                    Hm[(size_t)(k + 1) * m + k] = hn;
                    if (hn > 0)
                        for (int64_t i = 0; i < n; ++i) V[k + 1][i] /= hn;
                    for (int j = 0; j < k; ++j) {   // previous rotations
                        const cd a = Hm[(size_t)j * m + k], bb = Hm[(size_t)(j + 1) * m + k];
                        Hm[(size_t)j * m + k] = cr[j] * a + sn[j] * bb;
                        Hm[(size_t)(j + 1) * m + k] = -std::conj(sn[j]) * a + cr[j] * bb;
                    }
                    double c;
                    cd s;
                    givens(Hm[(size_t)k * m + k], Hm[(size_t)(k + 1) * m + k], c, s);
                    cr[k] = c;
                    sn[k] = s;
                    Hm[(size_t)k * m + k] = c * Hm[(size_t)k * m + k] + s * Hm[(size_t)(k + 1) * m + k];
                    Hm[(size_t)(k + 1) * m + k] = 0.0;
                    g[k + 1] = -std::conj(s) * g[k];
                    g[k] = c * g[k];
                    if (std::abs(g[k + 1]) <= target || used >= maxit) {
                        ++k;
                        break;
                    }
                }
                // y = H^-1 g; d += P V y
                std::vector<cd> y(k);
                for (int i = k - 1; i >= 0; --i) {
                    cd s = g[i];
                    for (int j = i + 1; j < k; ++j) s -= Hm[(size_t)i * m + j] * y[j];
                    y[i] = s / Hm[(size_t)i * m + i];
                }
                parallel_segments(n, [&](int, int64_t i0, int64_t i1) {
                    for (int64_t i = i0; i < i1; ++i) t[i] = 0.0;
                    for (int j = 0; j < k; ++j) {
                        const cd yj = y[j];
                        const cd *v = V[j].data();
                        for (int64_t i = i0; i < i1; ++i) t[i] += yj * v[i];
                    }
                });
                if (sai) sai->apply(t.data(), z.data());
                else z = t;
                for (int64_t i = 0; i < n; ++i) d[i] += z[i];
                // true residual of the inner system in the product precision
                mlfma_status st = prod->apply(which, d.data(), t.data(), prec);
                if (st) return st;
                for (int64_t i = 0; i < n; ++i) rr[i] = r[i] - t[i];
                rn = nrm2(rr);
            }
            for (int64_t i = 0; i < n; ++i) w[i] += d[i];
            // residual check with the checking precision (FP64 when available)
            mlfma_status st = prod->apply(which, w.data(), t.data(), check_prec);
            if (st) return st;
            for (int64_t i = 0; i < n; ++i) r[i] = b[i] - t[i];
            if (nrm2(r) <= tol * bn) {
                converged = true;
                break;
            }
        }
        return MLFMA_OK;
    }
};

}  // namespace

extern "C" mlfma_status mlfma_cm_default_opts(mlfma_cm_opts *o)
{
    if (!o) return fail(MLFMA_EINVAL, "opts is NULL");
    o->nev = 10;
    o->ncv = 30;
    o->op = MLFMA_CM_ZINV_R;
    o->prec = MLFMA_FP32;
    o->tol = 1e-8;
    o->gmres_tol = 1e-6;
    o->gmres_restart = 50;
    o->max_inner = 2000;
    o->max_restarts = 200;
    o->use_sai = 1;
    o->seed = 1412175602ULL;
    return MLFMA_OK;
}

extern "C" mlfma_status cm_ira_solve(mlfma_plan_t plan, const mlfma_cm_opts *opts, double *lambda, double *J,
                                     mlfma_cm_stats *stats)
{
    auto t0 = std::chrono::steady_clock::now();
    if (!plan || !opts || !lambda) return fail(MLFMA_EINVAL, "plan, opts and lambda are required");
    mlfma_cm_opts o = *opts;
    int64_t n = 0;
    if (mlfma_num_unknowns(plan, &n)) return MLFMA_EINVAL;
    if (o.nev < 1 || o.ncv <= o.nev + 1 || o.ncv > n) return fail(MLFMA_EINVAL, "need 1 <= nev < ncv - 1 and ncv <= N");
    if (o.op != MLFMA_CM_ZINV_R && o.op != MLFMA_CM_XINV_R) return fail(MLFMA_EINVAL, "unknown operator");
    if (o.prec != MLFMA_FP32 && o.prec != MLFMA_FP64) return fail(MLFMA_EINVAL, "unknown precision");
    if (!(o.tol > 0) || !(o.gmres_tol > 0) || o.gmres_restart < 2 || o.max_inner < 1 || o.max_restarts < 1)
        return fail(MLFMA_EINVAL, "bad tolerance or iteration limits");
    std::vector<cd> near;
    const PlanHost *H = nullptr;
    if (!plan_near_host(plan, near, &H)) return fail(MLFMA_EINVAL, "plan is host-only or its near field is unreadable");
    const bool has64 = [&]() {   // can the residual be checked in FP64?
        std::vector<double> x(2 * n, 0.0), y(4 * n);
        return mlfma_matvec_host(plan, x.data(), 1, y.data(), 1, MLFMA_FP64, nullptr) == MLFMA_OK;
    }();
    Products prod{plan, n, o.prec};
    Sai sai;
    if (o.use_sai && !sai.build(H, near, o.op == MLFMA_CM_XINV_R))
        return fail(MLFMA_ENOTCONV, "sparse approximate inverse: a near-field block is singular");
    near.clear();
    near.shrink_to_fit();
    Gmres gm{&prod, o.use_sai ? &sai : nullptr, o.op == MLFMA_CM_ZINV_R ? PROD_Z : PROD_X, o.prec,
             o.gmres_restart, o.max_inner, has64 ? MLFMA_FP64 : o.prec, o.gmres_tol};
    std::unique_ptr<DeviceGmres, void (*)(DeviceGmres *)> dgm(nullptr, device_gmres_destroy);
    if (o.prec == MLFMA_FP32) {   // FP32 inner passes on the device
        std::string err;
        dgm.reset(device_gmres_create(plan, o.use_sai ? sai.vals.data() : nullptr, o.gmres_restart, err));
        if (!dgm) return fail(MLFMA_ECUDA, err);
        gm.dev = dgm.get();
    }

    // the operator of Eq. (SEP1) or (SEP)
    std::vector<cd> tmp(n), rhs(n), sol(n);
    bool inner_ok = true;
    auto op = [&](const cd *v, cd *out) -> mlfma_status {
        mlfma_status st;
        bool conv = false;
        if (o.op == MLFMA_CM_ZINV_R) {
            // Z_H^-1 R v = conj(Zp^-1 (-R conj v))
            for (int64_t i = 0; i < n; ++i) tmp[i] = std::conj(v[i]);
            if ((st = prod.apply(PROD_R, tmp.data(), rhs.data(), o.prec))) return st;
            for (int64_t i = 0; i < n; ++i) rhs[i] = -rhs[i];
            if ((st = gm.solve(rhs, sol, conv))) return st;
            for (int64_t i = 0; i < n; ++i) out[i] = std::conj(sol[i]);
        } else {
            if ((st = prod.apply(PROD_R, v, rhs.data(), o.prec))) return st;
            if ((st = gm.solve(rhs, sol, conv))) return st;
            for (int64_t i = 0; i < n; ++i) out[i] = sol[i];
        }
        inner_ok = inner_ok && conv;
        return MLFMA_OK;
    };

    // the Arnoldi basis V_0..V_m lives on the device (FP64); the host keeps the
    // vector the next operator application needs and the Hessenberg matrix
    const int m = o.ncv, k = o.nev;
    std::string derr;
    std::unique_ptr<DeviceArnoldi, void (*)(DeviceArnoldi *)> arn(arnoldi_create(plan, n, m, derr), arnoldi_destroy);
    if (!arn) return fail(MLFMA_ECUDA, derr);
    std::vector<cd> vj(n), wv(n), hcol(m + 1);
    std::vector<cd> Hm((size_t)(m + 1) * m, 0.0);   // (m+1) x m, row-major
    std::mt19937_64 rng(o.seed);
    std::normal_distribution<double> nd(0.0, 1.0);
    for (int64_t i = 0; i < n; ++i) vj[i] = nd(rng);
    {
        const double v0 = nrm2(vj);
        for (auto &z : vj) z /= v0;
    }
    if (!arnoldi_set(arn.get(), 0, vj.data(), derr)) return fail(MLFMA_ECUDA, derr);
    int kstart = 0, restarts = 0;
    bool converged = false;
    std::vector<cd> w, X;
    std::vector<int> order;
    mlfma_status st;
    for (; restarts < o.max_restarts; ++restarts) {
        for (int j = kstart; j < m; ++j) {   // extend the Arnoldi factorisation to m steps
            if ((st = op(vj.data(), wv.data()))) return st;
            std::fill(hcol.begin(), hcol.end(), cd(0.0));
            double hn = 0;
            if (!arnoldi_extend(arn.get(), j, wv.data(), hcol.data(), &hn, j + 1 < m ? vj.data() : nullptr, derr))
                return fail(MLFMA_ECUDA, derr);
            for (int i = 0; i <= j; ++i) Hm[(size_t)i * m + j] += hcol[i];
            Hm[(size_t)(j + 1) * m + j] = hn;
        }
        std::vector<cd> Hsq(Hm.begin(), Hm.begin() + (size_t)m * m);
        if (!hessenberg_eig(m, Hsq, w, X)) return fail(MLFMA_ENOTCONV, "Hessenberg eigenvalue iteration failed");
        order.resize(m);
        for (int i = 0; i < m; ++i) order[i] = i;
        std::sort(order.begin(), order.end(), [&](int a2, int b2) { return std::abs(w[a2]) > std::abs(w[b2]); });
        const double beta = std::abs(Hm[(size_t)m * m + (m - 1)]);
        converged = true;
        for (int i = 0; i < k; ++i) {
            const int e = order[i];
            const double res = beta * std::abs(X[(size_t)(m - 1) * m + e]);
            if (res > o.tol * std::max(std::abs(w[e]), 1e-300)) converged = false;
        }
        if (converged || restarts + 1 == o.max_restarts) break;
        // implicit restart with the m - k unwanted Ritz values as shifts
        std::vector<cd> Q((size_t)m * m, 0.0);
        for (int i = 0; i < m; ++i) Q[(size_t)i * m + i] = 1.0;
        std::vector<cd> Hw(Hm.begin(), Hm.begin() + (size_t)m * m);
        for (int i = k; i < m; ++i) qr_sweep(m, Hw, Q, 0, m - 1, w[order[i]]);
        // V_j <- V Q e_j (j < k);  V_k <- f_k = V Q e_k * H+(k, k-1) + V_m * H(m, m-1) Q(m-1, k-1),
        // normalised: one recombination of the old basis on the device
        const cd hk = Hw[(size_t)k * m + (k - 1)], fm = Hm[(size_t)m * m + (m - 1)] * Q[(size_t)(m - 1) * m + (k - 1)];
        std::vector<cd> coef((size_t)(m + 1) * (k + 1), 0.0);
        for (int i = 0; i < m; ++i)
            for (int c = 0; c <= k; ++c) coef[(size_t)i * (k + 1) + c] = Q[(size_t)i * m + c] * (c == k ? hk : cd(1.0));
        coef[(size_t)m * (k + 1) + k] = fm;
        if (!arnoldi_recombine(arn.get(), m + 1, k + 1, coef.data(), derr)) return fail(MLFMA_ECUDA, derr);
        double fn = 0;
        if (!arnoldi_normalise(arn.get(), k, &fn, derr)) return fail(MLFMA_ECUDA, derr);
        std::fill(Hm.begin(), Hm.end(), 0.0);
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < k; ++j) Hm[(size_t)i * m + j] = Hw[(size_t)i * m + j];
        Hm[(size_t)k * m + (k - 1)] = fn;
        if (!arnoldi_get(arn.get(), k, vj.data(), derr)) return fail(MLFMA_ECUDA, derr);
        kstart = k;
    }
    // Ritz pairs -> characteristic values and real currents
    std::vector<std::pair<double, int>> lam;
    for (int i = 0; i < k; ++i) {
        const cd mu = w[order[i]];
        const double l = o.op == MLFMA_CM_ZINV_R ? ((1.0 / mu - 1.0) / cd(0, 1)).real() : (1.0 / mu).real();
        lam.push_back({l, order[i]});
    }
    std::sort(lam.begin(), lam.end(), [](const auto &a2, const auto &b2) { return std::abs(a2.first) < std::abs(b2.first); });
    for (int i = 0; i < k; ++i) lambda[i] = lam[i].first;
    if (J) {
        // Ritz vectors V X e (the wanted columns in output order) on the device
        std::vector<cd> coef((size_t)m * k), vs((size_t)k * n);
        for (int j = 0; j < m; ++j)
            for (int i = 0; i < k; ++i) coef[(size_t)j * k + i] = X[(size_t)j * m + lam[i].second];
        if (!arnoldi_combine(arn.get(), m, k, coef.data(), vs.data(), derr)) return fail(MLFMA_ECUDA, derr);
        for (int i = 0; i < k; ++i) {
            const cd *v = vs.data() + (size_t)i * n;
            // characteristic currents are real up to a phase: rotate to the
            // phase that maximises the real part's norm, normalise
            cd s2 = 0;
            for (int64_t r = 0; r < n; ++r) s2 += v[r] * v[r];
            const cd ph = std::polar(1.0, -0.5 * std::arg(s2));
            double nn = 0;
            for (int64_t r = 0; r < n; ++r) nn += std::pow((v[r] * ph).real(), 2);
            nn = std::sqrt(nn);
            for (int64_t r = 0; r < n; ++r) J[r * k + i] = (v[r] * ph).real() / nn;
        }
    }
    if (stats) {
        stats->restarts = restarts;
        stats->inner_iterations = gm.iterations;
        stats->products = prod.count;
        stats->converged = converged ? 1 : 0;
        stats->inner_converged = inner_ok ? 1 : 0;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    if (!converged) return fail(MLFMA_ENOTCONV, "Arnoldi did not converge within max_restarts");
    return MLFMA_OK;
}

// ------------------------------------------ block subspace iteration ---

extern "C" mlfma_status cm_rayleigh_ritz(int64_t n, int p, const double *Y, const double *RY, const double *W,
                                         double *mu, double *coef, int *rank)
{
    if (n < 1 || p < 1 || !Y || !RY || !W || !mu || !coef || !rank)
        return fail(MLFMA_EINVAL, "cm_rayleigh_ritz: NULL argument or empty block");
    std::vector<double> m, c;
    const int r = ritz_shift_invert(n, p, Y, RY, W, m, c);
    for (int i = 0; i < p; ++i) mu[i] = i < r ? m[i] : 0.0;
    for (int a = 0; a < p; ++a)
        for (int i = 0; i < p; ++i) coef[(size_t)a * p + i] = i < r ? c[(size_t)a * r + i] : 0.0;
    *rank = r;
    return MLFMA_OK;
}

// Eq. (SEP) with a block of ncv vectors: shift-invert subspace iteration
// (simultaneous iteration, Rutishauser 1970) on T = X^-1 R.  Every
// iteration solves X W = R Y for the whole block at once (block_gmres_run:
// one product of ncv real columns per GMRES step), takes the Ritz pairs of T
// on span Y in the R inner product (ritz_shift_invert: A = (R Y)^T W,
// B = Y^T R Y), and moves to the improved vectors Y' = W coef, applying Z to
// Y' once (X Y' and R Y' are its imaginary and negated real parts).  The
// reported values are the Rayleigh quotients y^T X y / y^T R y of the final
// vectors (second order in their error).  A degenerate cluster that fits in
// the block converges as a whole, which a single-vector Krylov method
// cannot resolve; errors of the inexact solves along near-null vectors of X
// (interior resonances: currents that do not radiate) are filtered by R.
// With MLFMA_CM_TRACE set in the environment, one line per iteration goes to
// stderr (MLFMA_CM_TRACE=2: also one per wanted column).
extern "C" mlfma_status cm_block_solve(mlfma_plan_t plan, const mlfma_cm_opts *opts, double *lambda, double *J,
                                       mlfma_cm_stats *stats)
{
    auto t0 = std::chrono::steady_clock::now();
    if (!plan || !opts || !lambda) return fail(MLFMA_EINVAL, "plan, opts and lambda are required");
    const mlfma_cm_opts o = *opts;
    int dev = 0, maxb = 0;
    int64_t n = 0;
    if (!plan_product_view(plan, MLFMA_FP32, 0, nullptr, nullptr, &dev, &maxb, &n))
        return fail(MLFMA_EINVAL, "cm_block_solve needs a device plan with FP32 products");
    const int p = o.ncv, k = o.nev;
    if (k < 1 || p < k || p > n || p > maxb) return fail(MLFMA_EINVAL, "need 1 <= nev <= ncv <= min(N, max_batch)");
    if (o.op != MLFMA_CM_XINV_R) return fail(MLFMA_EINVAL, "the block solver works on X^-1 R (MLFMA_CM_XINV_R)");
    if (o.prec != MLFMA_FP32 && o.prec != MLFMA_FP64) return fail(MLFMA_EINVAL, "unknown precision");
    if (!(o.gmres_tol > 0) || !(o.tol > 0) || o.gmres_restart < 1 || o.max_inner < 1 || o.max_restarts < 1)
        return fail(MLFMA_EINVAL, "bad tolerance or iteration limits");
    const char *trace_env = std::getenv("MLFMA_CM_TRACE");
    const int trace = trace_env ? std::max(1, std::atoi(trace_env)) : 0;   // 2: every column as well
    std::vector<cd> near;
    const PlanHost *H = nullptr;
    if (!plan_near_host(plan, near, &H)) return fail(MLFMA_EINVAL, "plan is host-only or its near field is unreadable");
    Sai sai;
    if (o.use_sai && !sai.build(H, near, true))
        return fail(MLFMA_ENOTCONV, "sparse approximate inverse: a near-field block is singular");
    near.clear();
    near.shrink_to_fit();
    std::string err;
    std::unique_ptr<BlockGmres, void (*)(BlockGmres *)> bg(
        block_gmres_create(plan, o.use_sai ? sai.vals.data() : nullptr, o.gmres_restart, p, err), block_gmres_destroy);
    if (!bg) return fail(MLFMA_ECUDA, err);

    const size_t np = (size_t)n * p;
    int64_t nprod = 0, inner = 0;
    std::vector<float> xf, yf;
    std::vector<double> yd;
    // X Y = Im(Zp Y), R Y = -Re(Zp Y) for the p real columns of Y (one product)
    auto products = [&](const std::vector<double> &Yb, std::vector<double> &XY, std::vector<double> &RY) {
        mlfma_status st;
        if (o.prec == MLFMA_FP32) {
            xf.resize(np);
            yf.resize(2 * np);
            for (size_t e = 0; e < np; ++e) xf[e] = (float)Yb[e];
            if ((st = mlfma_matvec_host(plan, xf.data(), 0, yf.data(), p, MLFMA_FP32, nullptr))) return st;
            for (size_t e = 0; e < np; ++e) {
                XY[e] = yf[2 * e + 1];
                RY[e] = -(double)yf[2 * e];
            }
        } else {
            yd.resize(2 * np);
            if ((st = mlfma_matvec_host(plan, Yb.data(), 0, yd.data(), p, MLFMA_FP64, nullptr))) return st;
            for (size_t e = 0; e < np; ++e) {
                XY[e] = yd[2 * e + 1];
                RY[e] = -yd[2 * e];
            }
        }
        ++nprod;
        return MLFMA_OK;
    };
    auto normalise_columns = [&](std::vector<double> &Yb) {
        std::vector<double> nn(p, 0.0);
        for (size_t e = 0; e < np; ++e) nn[e % p] += Yb[e] * Yb[e];
        for (int c = 0; c < p; ++c) nn[c] = nn[c] > 0 ? 1 / std::sqrt(nn[c]) : 0.0;
        for (size_t e = 0; e < np; ++e) Yb[e] *= nn[e % p];
    };
    std::mt19937_64 rng(o.seed);
    std::normal_distribution<double> nd(0.0, 1.0);
    std::vector<double> Y(np), XY(np), RY(np), W(np), Yn(np), mu, coef, relres(p);
    for (auto &v : Y) v = nd(rng);
    normalise_columns(Y);
    mlfma_status st;
    if ((st = products(Y, XY, RY))) return st;
    std::vector<int> conv(p), order(p);
    for (int c = 0; c < p; ++c) order[c] = c;
    std::vector<double> lam(p, INFINITY), res(p, INFINITY);
    bool converged = false, inner_ok = true;
    int iters = 0;
    while (iters < o.max_restarts) {
        ++iters;
        // initial guess X^-1 R y = y / lambda for the columns that hold
        // Ritz pairs with residual below 0.1 (zero elsewhere and on the first
        // iteration): it carries the large components along the wanted
        // modes, the near-null vectors of X that GMRES resolves last; for a
        // poor pair the guess's own residual (X y - lambda R y) / lambda
        // would exceed that of zero
        for (int64_t q = 0; q < n; ++q)
            for (int c = 0; c < p; ++c) {
                const size_t e = (size_t)q * p + c;
                W[e] = std::isfinite(lam[c]) && lam[c] != 0 && res[c] < 0.1 ? Y[e] / lam[c] : 0.0;
            }
        const int used = block_gmres_run(bg.get(), RY.data(), W.data(), 1, o.gmres_tol, o.max_inner, conv.data(),
                                         relres.data(), err);
        if (used < 0) return fail(MLFMA_ECUDA, err);
        inner += used;
        nprod += used;
        for (int c = 0; c < p; ++c) inner_ok = inner_ok && conv[c];
        const int r = ritz_shift_invert(n, p, Y.data(), RY.data(), W.data(), mu, coef);
        if (r < 1) return fail(MLFMA_ENOTCONV, "block solver: the block lost all R energy");
        // next block: the r improved Ritz vectors W coef, random directions
        // in the columns the block lost; one product gives X Y' and R Y'
        right_multiply(n, p, r, W.data(), coef, XY.data());   // XY as scratch [n][r]
        for (int64_t q = 0; q < n; ++q)
            for (int c = 0; c < p; ++c) Yn[(size_t)q * p + c] = c < r ? XY[(size_t)q * r + c] : nd(rng);
        normalise_columns(Yn);
        Y.swap(Yn);
        if ((st = products(Y, XY, RY))) return st;
        // Rayleigh quotients lambda = y^T X y / y^T R y and residuals
        // ||X y - lambda R y|| / (||X y|| + |lambda| ||R y||) of the columns
        std::vector<double> yx(p, 0.0), yr(p, 0.0), xx(p, 0.0), rr2(p, 0.0), xr(p, 0.0);
        for (int64_t q = 0; q < n; ++q)
            for (int c = 0; c < p; ++c) {
                const size_t e = (size_t)q * p + c;
                yx[c] += Y[e] * XY[e];
                yr[c] += Y[e] * RY[e];
                xx[c] += XY[e] * XY[e];
                rr2[c] += RY[e] * RY[e];
                xr[c] += XY[e] * RY[e];
            }
        for (int c = 0; c < p; ++c) {
            lam[c] = c < r && yr[c] > 0 ? yx[c] / yr[c] : INFINITY;
            if (!std::isfinite(lam[c])) {
                res[c] = INFINITY;
                continue;
            }
            const double d2 = xx[c] - 2 * lam[c] * xr[c] + lam[c] * lam[c] * rr2[c];
            res[c] = std::sqrt(std::max(0.0, d2)) / (std::sqrt(xx[c]) + std::abs(lam[c]) * std::sqrt(rr2[c]) + 1e-300);
        }
        // the wanted pairs are the first nev columns: Ritz order, largest
        // |mu| first.  Interlacing makes that order safe; the Rayleigh
        // quotient of an unconverged vector under an indefinite X is not
        // (the block's last columns can have quotients near zero), so it
        // reports values but does not select them.  Output in |lambda| order.
        for (int c = 0; c < p; ++c) order[c] = c;
        std::stable_sort(order.begin(), order.begin() + std::min(k, p),
                         [&](int x, int y) { return std::abs(lam[x]) < std::abs(lam[y]); });
        converged = r >= k;
        double worst = 0, worst_inner = 0;
        for (int i = 0; i < k; ++i) {
            worst = std::max(worst, res[order[i]]);
            if (!(res[order[i]] <= o.tol)) converged = false;
        }
        for (int c = 0; c < p; ++c) worst_inner = std::max(worst_inner, relres[c]);
        if (trace)
            std::fprintf(stderr, "cm_block_solve: iteration %d  GMRES steps %d  max inner residual %.2e  rank %d  "
                         "max residual of the %d wanted %.2e  lambda_1 %.8g  %.1f s\n", iters, used, worst_inner, r, k,
                         worst, lam[order[0]], std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count());
        if (trace >= 2)
            for (int i = 0; i < std::min(p, k + 6); ++i) {
                const int c = order[i];
                std::fprintf(stderr, "  column %2d  Rayleigh quotient %+.8f  Ritz 1/mu %+.8f  residual %.2e  inner %.2e\n",
                             c, lam[c], c < r ? 1.0 / mu[c] : INFINITY, res[c], relres[c]);
            }
        if (converged) break;
    }
    for (int i = 0; i < k; ++i) lambda[i] = std::isfinite(lam[order[i]]) ? lam[order[i]] : std::nan("");
    if (J) {
        for (int i = 0; i < k; ++i) {
            const int c = order[i];
            double nn = 0, big = 0;
            for (int64_t q = 0; q < n; ++q) {
                const double v = Y[(size_t)q * p + c];
                nn += v * v;
                if (std::abs(v) > std::abs(big)) big = v;
            }
            const double f = nn > 0 ? (big < 0 ? -1.0 : 1.0) / std::sqrt(nn) : 0.0;   // unit norm, largest entry > 0
            for (int64_t q = 0; q < n; ++q) J[q * k + i] = f * Y[(size_t)q * p + c];
        }
    }
    if (stats) {
        stats->restarts = iters;
        stats->inner_iterations = inner;
        stats->products = nprod;
        stats->converged = converged ? 1 : 0;
        stats->inner_converged = inner_ok ? 1 : 0;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    if (!converged) return fail(MLFMA_ENOTCONV, "block subspace iteration did not converge within max_restarts");
    return MLFMA_OK;
}

// ----------------------------------------- characteristic-value slopes ---

// d lambda / dk of characteristic pairs (Section II, Eq. (GEP), with the
// pencil's k-derivative): for X J = lambda R J with R = -Re Z, X = Im Z and
// a real J,  d lambda/dk = J^T (X' - lambda R') J / (J^T R J),  where
// X' J = Im(Z' J), R' J = -Re(Z' J) and R J = -Re(Z J) come from one
// mlfma_matvec_dk and one mlfma_matvec per column (GPU, `prec`); the dot
// products are FP64 on the host.
extern "C" mlfma_status cm_eig_derivatives(mlfma_plan_t plan, int nev, const double *lambda, const double *J,
                                           int prec, double *dlambda)
{
    if (!plan || !lambda || !J || !dlambda || nev < 1) return fail(MLFMA_EINVAL, "NULL argument or nev < 1");
    int dev = 0, max_batch = 0;
    int64_t n = 0;
    if (!plan_product_view(plan, prec, 0, nullptr, nullptr, &dev, &max_batch, &n))
        return fail(MLFMA_EINVAL, "plan is host-only or the precision is not set up");
    const int chunk = std::max(1, max_batch / 2);
    const size_t rsz = prec == MLFMA_FP64 ? 8 : 4;
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
    void *dx = nullptr, *dz = nullptr, *dd = nullptr;
    mlfma_status st = MLFMA_OK;
    cudaError_t e = cudaMalloc(&dx, (size_t)n * chunk * rsz);
    if (e == cudaSuccess) e = cudaMalloc(&dz, (size_t)n * chunk * 2 * rsz);
    if (e == cudaSuccess) e = cudaMalloc(&dd, (size_t)n * chunk * 2 * rsz);
    if (e != cudaSuccess) st = fail(MLFMA_ENOMEM, "cm_eig_derivatives: device buffers");
    std::vector<char> hx((size_t)n * chunk * rsz), hz((size_t)n * chunk * 2 * rsz), hd(hz.size());
    for (int c0 = 0; c0 < nev && st == MLFMA_OK; c0 += chunk) {
        const int cb = std::min(chunk, nev - c0);
        for (int64_t r = 0; r < n; ++r)
            for (int c = 0; c < cb; ++c) {
                const double v = J[r * nev + c0 + c];
                if (prec == MLFMA_FP64) reinterpret_cast<double *>(hx.data())[r * cb + c] = v;
                else reinterpret_cast<float *>(hx.data())[r * cb + c] = (float)v;
            }
        if ((e = cudaMemcpy(dx, hx.data(), (size_t)n * cb * rsz, cudaMemcpyHostToDevice)) != cudaSuccess) {
            st = fail(MLFMA_ECUDA, std::string("cm_eig_derivatives: ") + cudaGetErrorString(e));
            break;
        }
        if ((st = mlfma_matvec(plan, dx, 0, dz, cb, prec, nullptr)) != MLFMA_OK) break;
        if ((st = mlfma_matvec_dk(plan, dx, 0, dd, cb, prec, nullptr)) != MLFMA_OK) break;
        if ((e = cudaMemcpy(hz.data(), dz, (size_t)n * cb * 2 * rsz, cudaMemcpyDeviceToHost)) != cudaSuccess ||
            (e = cudaMemcpy(hd.data(), dd, (size_t)n * cb * 2 * rsz, cudaMemcpyDeviceToHost)) != cudaSuccess) {
            st = fail(MLFMA_ECUDA, std::string("cm_eig_derivatives: ") + cudaGetErrorString(e));
            break;
        }
        auto val = [&](const std::vector<char> &h, int64_t r, int c, int part) -> double {
            const size_t i = ((size_t)r * cb + c) * 2 + part;
            return prec == MLFMA_FP64 ? reinterpret_cast<const double *>(h.data())[i]
                                      : (double)reinterpret_cast<const float *>(h.data())[i];
        };
        for (int c = 0; c < cb; ++c) {
            double jrj = 0, jxd = 0, jrd = 0;
            for (int64_t r = 0; r < n; ++r) {
                const double j = J[r * nev + c0 + c];
                jrj -= j * val(hz, r, c, 0);
                jxd += j * val(hd, r, c, 1);
                jrd -= j * val(hd, r, c, 0);
            }
            dlambda[c0 + c] = (jxd - lambda[c0 + c] * jrd) / jrj;
        }
    }
    cudaFree(dx);
    cudaFree(dz);
    cudaFree(dd);
    if (prev != dev) cudaSetDevice(prev);
    return st;
}

// ------------------------------------------------- modes over frequency ---

// Matching the modes of one wavenumber to those of the previous one, by
// their currents (the paper follows characteristic values over frequency in
// Section V without saying how modes are paired).  The currents of a
// degenerate cluster span a subspace whose basis the eigensolver picks
// freely, so clusters are paired first, by how much of one cluster's span
// lies in the other's, and single modes inside paired clusters afterwards.
//   1. columns scaled to unit 2-norm; clusters: runs of values (sorted)
//      whose neighbours differ by at most cluster_tol * max(|lambda|, 1e-12);
//   2. cluster score s(A, B) = ||Ja_A^T Jb_B||_F^2 / min(|A|, |B|) (1 when
//      the smaller span lies in the larger), pairs taken greedily by
//      decreasing score while s >= 0.5, each cluster once;
//   3. inside a pair, modes matched greedily by |Ja_i . Jb_j|.
extern "C" mlfma_status cm_track_modes(int64_t n, int na, const double *lambda_a, const double *Ja, int nb,
                                       const double *lambda_b, const double *Jb, double cluster_tol, int *match,
                                       double *overlap)
{
    if (n < 1 || na < 1 || nb < 1 || !lambda_a || !Ja || !lambda_b || !Jb || !match || !overlap || !(cluster_tol >= 0))
        return fail(MLFMA_EINVAL, "cm_track_modes: NULL argument, empty set or negative cluster_tol");
    auto norms = [&](const double *J, int m) {
        std::vector<double> s(m, 0.0);
        for (int64_t r = 0; r < n; ++r)
            for (int c = 0; c < m; ++c) s[c] += J[r * m + c] * J[r * m + c];
        for (double &v : s) v = v > 0 ? 1.0 / std::sqrt(v) : 0.0;
        return s;
    };
    const std::vector<double> sa = norms(Ja, na), sb = norms(Jb, nb);
    // O[i][j] = Ja_i . Jb_j (unit columns)
    std::vector<double> O((size_t)na * nb, 0.0);
    for (int64_t r = 0; r < n; ++r)
        for (int i = 0; i < na; ++i) {
            const double a = Ja[r * na + i] * sa[i];
            if (a == 0.0) continue;
            for (int j = 0; j < nb; ++j) O[(size_t)i * nb + j] += a * Jb[r * nb + j];
        }
    for (int i = 0; i < na; ++i)
        for (int j = 0; j < nb; ++j) O[(size_t)i * nb + j] *= sb[j];
    auto clusters = [&](const double *lam, int m) {
        std::vector<int> ord(m);
        for (int i = 0; i < m; ++i) ord[i] = i;
        std::sort(ord.begin(), ord.end(), [&](int x, int y) { return lam[x] < lam[y]; });
        std::vector<std::vector<int>> cl;
        for (int t = 0; t < m; ++t) {
            const int i = ord[t];
            if (t > 0) {
                const double p = lam[ord[t - 1]];
                if (std::fabs(lam[i] - p) <= cluster_tol * std::max({std::fabs(lam[i]), std::fabs(p), 1e-12})) {
                    cl.back().push_back(i);
                    continue;
                }
            }
            cl.push_back({i});
        }
        return cl;
    };
    const auto ca = clusters(lambda_a, na), cb = clusters(lambda_b, nb);
    struct Pair {
        double s;
        int a, b;
    };
    std::vector<Pair> pairs;
    for (int x = 0; x < (int)ca.size(); ++x)
        for (int y = 0; y < (int)cb.size(); ++y) {
            double f = 0;
            for (int i : ca[x])
                for (int j : cb[y]) f += O[(size_t)i * nb + j] * O[(size_t)i * nb + j];
            pairs.push_back({f / (double)std::min(ca[x].size(), cb[y].size()), x, y});
        }
    std::sort(pairs.begin(), pairs.end(), [](const Pair &u, const Pair &v) { return u.s > v.s; });
    std::vector<char> used_a(ca.size(), 0), used_b(cb.size(), 0);
    for (int j = 0; j < nb; ++j) {
        match[j] = -1;
        overlap[j] = 0.0;
    }
    for (const Pair &pr : pairs) {
        if (pr.s < 0.5) break;
        if (used_a[pr.a] || used_b[pr.b]) continue;
        used_a[pr.a] = used_b[pr.b] = 1;
        std::vector<int> ia = ca[pr.a], ib = cb[pr.b];
        while (!ia.empty() && !ib.empty()) {
            size_t bi = 0, bj = 0;
            double best = -1;
            for (size_t u = 0; u < ia.size(); ++u)
                for (size_t v = 0; v < ib.size(); ++v) {
                    const double o = std::fabs(O[(size_t)ia[u] * nb + ib[v]]);
                    if (o > best) { best = o; bi = u; bj = v; }
                }
            match[ib[bj]] = ia[bi];
            ia.erase(ia.begin() + bi);
            ib.erase(ib.begin() + bj);
        }
        for (int j : cb[pr.b]) overlap[j] = std::min(1.0, pr.s);
    }
    return MLFMA_OK;
}
