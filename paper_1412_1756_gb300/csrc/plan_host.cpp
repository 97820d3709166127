// Host-side plan construction (FP64).  See plan_host.h.
#include "plan_host.h"

#include <algorithm>
#include <cmath>
#include <numeric>
#include <unordered_map>

namespace mlfma {

static const double kPi = 3.14159265358979323846;
static const int kWinMax = 32;   // widest window of the windowed stencil tables

// ------------------------------------------------------------ specfun ---
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w)
{
    // Newton iteration on P_n from the asymptotic guess; nodes descend.
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
        double pn = 0, pm = 0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int m = 2; m <= n; ++m) {
                double p2 = ((2.0 * m - 1.0) * z * p1 - (m - 1.0) * p0) / m;
                p0 = p1;
                p1 = p2;
            }
            pn = p1;
            pm = p0;
            double dp = n * (z * pn - pm) / (z * z - 1.0);
            double dz = pn / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int m = 2; m <= n; ++m) {
            double p2 = ((2.0 * m - 1.0) * z * p1 - (m - 1.0) * p0) / m;
            p0 = p1;
            p1 = p2;
        }
        double dp = (n == 1) ? 1.0 : n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

void sph_bessel_y(int nmax, double x, std::vector<double> &y)
{
    // upward recurrence y_{n+1} = (2n+1)/x y_n - y_{n-1}, stable for y
    y.assign(nmax + 1, 0.0);
    y[0] = -std::cos(x) / x;
    if (nmax >= 1) y[1] = -std::cos(x) / (x * x) - std::sin(x) / x;
    for (int n = 1; n < nmax; ++n) y[n + 1] = (2.0 * n + 1.0) / x * y[n] - y[n - 1];
}

void sph_bessel_j(int nmax, double x, std::vector<double> &j)
{
    // Miller's downward recurrence from well above max(nmax, x), then
    // normalised with whichever of j_0, j_1 is larger in magnitude.
    int start = std::max(nmax, (int)x) + 40 + (int)std::sqrt(40.0 * std::max((double)nmax, x));
    std::vector<double> f(start + 2, 0.0);
    f[start + 1] = 0.0;
    f[start] = 1e-300;
    for (int n = start; n > 0; --n) {
        f[n - 1] = (2.0 * n + 1.0) / x * f[n] - f[n + 1];
        if (std::fabs(f[n - 1]) > 1e250) {
            for (int m = n - 1; m <= start + 1; ++m) f[m] *= 1e-250;
        }
    }
    double j0 = std::sin(x) / x;
    double j1 = std::sin(x) / (x * x) - std::cos(x) / x;
    double s = (std::fabs(j0) >= std::fabs(j1)) ? j0 / f[0] : j1 / f[1];
    j.assign(nmax + 1, 0.0);
    for (int n = 0; n <= nmax; ++n) j[n] = f[n] * s;
}

int truncation_number(double k, double a, double digits)
{
    const double kd = k * std::sqrt(3.0) * a;
    const double L = kd + 1.8 * std::pow(digits, 2.0 / 3.0) * std::cbrt(kd);
    return std::max(1, (int)std::ceil(L - 1e-12));
}

// ------------------------------------------------------------- Morton ---
static uint64_t spread3(uint64_t v)
{
    v &= 0x1fffff;
    v = (v | v << 32) & 0x1f00000000ffffULL;
    v = (v | v << 16) & 0x1f0000ff0000ffULL;
    v = (v | v << 8) & 0x100f00f00f00f00fULL;
    v = (v | v << 4) & 0x10c30c30c30c30c3ULL;
    v = (v | v << 2) & 0x1249249249249249ULL;
    return v;
}
static uint64_t compact3(uint64_t v)
{
    v &= 0x1249249249249249ULL;
    v = (v ^ (v >> 2)) & 0x10c30c30c30c30c3ULL;
    v = (v ^ (v >> 4)) & 0x100f00f00f00f00fULL;
    v = (v ^ (v >> 8)) & 0x1f0000ff0000ffULL;
    v = (v ^ (v >> 16)) & 0x1f00000000ffffULL;
    v = (v ^ (v >> 32)) & 0x1fffff;
    return v;
}
static uint64_t morton(uint64_t x, uint64_t y, uint64_t z) { return spread3(x) << 2 | spread3(y) << 1 | spread3(z); }
static void unmorton(uint64_t c, int64_t &x, int64_t &y, int64_t &z)
{
    x = (int64_t)compact3(c >> 2);
    y = (int64_t)compact3(c >> 1);
    z = (int64_t)compact3(c);
}

// --------------------------------------------------------- stencils ---
// Lagrange weights of `p` consecutive entries of the sorted periodic
// extension `pos` around target t.
static void window_weights(const std::vector<double> &pos, double t, int p, int &s, std::vector<double> &c)
{
    int i0 = (int)(std::upper_bound(pos.begin(), pos.end(), t) - pos.begin()) - 1;
    s = i0 - p / 2 + 1;
    s = std::max(0, std::min(s, (int)pos.size() - p));
    c.assign(p, 1.0);
    for (int e = 0; e < p; ++e)
        for (int f = 0; f < p; ++f)
            if (f != e) c[e] *= (t - pos[s + f]) / (pos[s + e] - pos[s + f]);
}

// theta: source nodes th_src (ascending, in (0, pi)); the theta component of
// a tangential field continues past the poles as F(-th, ph) = -F(th, ph+pi)
// and is 2 pi periodic, so the extension holds +-th_j + 2 pi m.
static void theta_stencil(const std::vector<double> &src, const std::vector<double> &tgt, int p, Stencil &S)
{
    struct Node { double pos; int idx; int refl; };
    std::vector<Node> ext;
    for (int m = -1; m <= 1; ++m)
        for (int j = 0; j < (int)src.size(); ++j) {
            ext.push_back({src[j] + 2 * kPi * m, j, 0});
            ext.push_back({-src[j] + 2 * kPi * m, j, 1});
        }
    std::sort(ext.begin(), ext.end(), [](const Node &a, const Node &b) { return a.pos < b.pos; });
    std::vector<double> pos(ext.size());
    for (size_t i = 0; i < ext.size(); ++i) pos[i] = ext[i].pos;
    S.ptr.assign(1, 0);
    S.idx.clear(); S.refl.clear(); S.coef.clear();
    std::vector<double> c;
    for (double t : tgt) {
        int s;
        window_weights(pos, t, p, s, c);
        for (int e = 0; e < p; ++e) {
            const Node &n = ext[s + e];
            S.idx.push_back(n.idx);
            S.refl.push_back(n.refl);
            S.coef.push_back(n.refl ? -c[e] : c[e]);
        }
        S.ptr.push_back((int32_t)S.idx.size());
    }
}

// phi: uniform periodic source grid of n points, targets ph_tgt.
static void phi_stencil(int n, const std::vector<double> &tgt, int p, Stencil &S)
{
    std::vector<double> pos;
    std::vector<int> idx;
    for (int m = -1; m <= 1; ++m)
        for (int v = 0; v < n; ++v) {
            pos.push_back(2 * kPi * v / n + 2 * kPi * m);
            idx.push_back(v);
        }
    S.ptr.assign(1, 0);
    S.idx.clear(); S.refl.clear(); S.coef.clear();
    std::vector<double> c;
    for (double t : tgt) {
        int s;
        window_weights(pos, t, p, s, c);
        for (int e = 0; e < p; ++e) {
            S.idx.push_back(idx[s + e]);
            S.refl.push_back(0);
            S.coef.push_back(c[e]);
        }
        S.ptr.push_back((int32_t)S.idx.size());
    }
}

// Transpose a stencil (nrows_src rows after transposition), scaling entries.
template <class Scale>
static void transpose_stencil(const Stencil &F, int nrows_out, Scale scale, Stencil &Tr)
{
    std::vector<std::vector<int>> rows(nrows_out);
    for (int r = 0; r + 1 < (int)F.ptr.size(); ++r)
        for (int e = F.ptr[r]; e < F.ptr[r + 1]; ++e) rows[F.idx[e]].push_back(e);
    Tr.ptr.assign(1, 0);
    Tr.idx.clear(); Tr.refl.clear(); Tr.coef.clear();
    std::vector<int> rowof(F.idx.size());
    for (int r = 0; r + 1 < (int)F.ptr.size(); ++r)
        for (int e = F.ptr[r]; e < F.ptr[r + 1]; ++e) rowof[e] = r;
    for (int j = 0; j < nrows_out; ++j) {
        for (int e : rows[j]) {
            Tr.idx.push_back(rowof[e]);
            Tr.refl.push_back(F.refl.empty() ? 0 : F.refl[e]);
            Tr.coef.push_back(F.coef[e] * scale(rowof[e], j));
        }
        Tr.ptr.push_back((int32_t)Tr.idx.size());
    }
}

// ------------------------------------------------------ windowed rows ---
bool win_stencil(const Stencil &S, int n, bool theta, int tw_max, WinStencil &W)
{
    const int rows = (int)S.ptr.size() - 1;
    W = WinStencil();
    if (rows <= 0 || n <= 0) return false;
    const int groups = (rows + kWinRows - 1) / kWinRows;
    struct Ent { int row, pos; double c; };
    std::vector<std::vector<Ent>> ent(groups);
    std::vector<int> lo(groups), hi(groups);
    int tw = 0;
    for (int g = 0; g < groups; ++g) {
        const int r0 = g * kWinRows, r1 = std::min(rows, r0 + kWinRows);
        if (theta) {
            for (int r = r0; r < r1; ++r) {
                // a reflected sample goes to the pole nearer the row's direct taps
                double sum = 0;
                int cnt = 0;
                for (int e = S.ptr[r]; e < S.ptr[r + 1]; ++e)
                    if (!S.refl[e]) { sum += S.idx[e]; ++cnt; }
                const double mid = cnt ? sum / cnt : (r < rows / 2 ? 0.0 : n - 1.0);
                for (int e = S.ptr[r]; e < S.ptr[r + 1]; ++e) {
                    int pos = S.idx[e];
                    if (S.refl[e]) {
                        const int north = -pos - 1, south = 2 * n - pos - 1;
                        pos = std::abs(north - mid) <= std::abs(south - mid) ? north : south;
                    }
                    ent[g].push_back({r - r0, pos, S.coef[e]});
                }
            }
        } else {
            // the shortest arc of the periodic grid holding every tap of the group
            std::vector<int> u;
            for (int r = r0; r < r1; ++r)
                for (int e = S.ptr[r]; e < S.ptr[r + 1]; ++e) u.push_back(S.idx[e]);
            std::sort(u.begin(), u.end());
            u.erase(std::unique(u.begin(), u.end()), u.end());
            int best = -1, gap = -1;
            for (size_t i = 0; i < u.size(); ++i) {
                const int nx = i + 1 < u.size() ? u[i + 1] : u[0] + n;
                if (nx - u[i] > gap) { gap = nx - u[i]; best = (int)i; }
            }
            const int st = u[(best + 1) % u.size()];
            for (int r = r0; r < r1; ++r)
                for (int e = S.ptr[r]; e < S.ptr[r + 1]; ++e)
                    ent[g].push_back({r - r0, st + ((S.idx[e] - st) % n + n) % n, S.coef[e]});
        }
        lo[g] = hi[g] = ent[g].front().pos;
        for (const Ent &x : ent[g]) { lo[g] = std::min(lo[g], x.pos); hi[g] = std::max(hi[g], x.pos); }
        tw = std::max(tw, hi[g] - lo[g] + 1);
        if (theta && (lo[g] < -n || hi[g] >= 2 * n)) return false;
    }
    if (tw > tw_max || (!theta && tw > n) || (theta && tw > 3 * n)) return false;
    W.groups = groups;
    W.tw = tw;
    W.start.resize(groups);
    W.coef.assign((size_t)groups * tw * kWinRows, 0.0);
    for (int g = 0; g < groups; ++g) {
        // theta: keep the window inside [-n, 2n); phi: start in [0, n)
        int st = lo[g];
        if (theta) st = std::max(-n, std::min(st, 2 * n - tw));
        for (const Ent &x : ent[g]) W.coef[((size_t)g * tw + (x.pos - st)) * kWinRows + x.row] += x.c;
        W.start[g] = theta ? st : ((st % n) + n) % n;
    }
    return true;
}

// ------------------------------------------------------------- grids ---
static void make_grid(Level &Lv, double k, double digits)
{
    Lv.L = truncation_number(k, Lv.a, digits);
    Lv.nth = Lv.L + 1;
    Lv.nph = 2 * (Lv.L + 1);
    Lv.K = Lv.nth * Lv.nph;
    std::vector<double> x, w;
    gauss_legendre(Lv.nth, x, w);
    Lv.ct = x;
    Lv.wt = w;
    Lv.th.resize(Lv.nth);
    for (int i = 0; i < Lv.nth; ++i) Lv.th[i] = std::acos(x[i]);
    Lv.ph.resize(Lv.nph);
    for (int j = 0; j < Lv.nph; ++j) Lv.ph[j] = 2 * kPi * j / Lv.nph;
}

static void khat(const Level &Lv, int q, double *kh)
{
    const int it = q / Lv.nph, ip = q % Lv.nph;
    const double st = std::sqrt(std::max(0.0, 1.0 - Lv.ct[it] * Lv.ct[it]));
    kh[0] = st * std::cos(Lv.ph[ip]);
    kh[1] = st * std::sin(Lv.ph[ip]);
    kh[2] = Lv.ct[it];
}

// Eq. (8): alpha(khat, r) = sum_{l=0}^{L} i^l (2l+1) h_l^(1)(k r) P_l(khat . rhat),
// and its k-derivative with the samples and L fixed: r h_l^(1)'(k r) in place
// of h_l^(1)(k r), where h_0' = -h_1 and h_l' = h_{l-1} - (l+1)/x h_l.
static void translation_table(Level &Lv, double k)
{
    Lv.alpha.assign((size_t)Lv.ntype * Lv.K, cd(0, 0));
    Lv.alpha_dk.assign((size_t)Lv.ntype * Lv.K, cd(0, 0));
    Lv.alpha_j.assign((size_t)Lv.ntype * Lv.K, cd(0, 0));
    Lv.alpha_y.assign((size_t)Lv.ntype * Lv.K, cd(0, 0));
    std::vector<double> jn, yn, jd, yd, P(Lv.L + 1);
    for (int t = 0; t < Lv.ntype; ++t) {
        double r[3] = {Lv.a * Lv.type_off[3 * t], Lv.a * Lv.type_off[3 * t + 1], Lv.a * Lv.type_off[3 * t + 2]};
        double rn = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        double x = k * rn;
        sph_bessel_j(Lv.L, x, jn);
        sph_bessel_y(Lv.L, x, yn);
        sph_bessel_j(Lv.L + 1, x, jd);
        sph_bessel_y(Lv.L + 1, x, yd);
        std::vector<cd> coef(Lv.L + 1), coefd(Lv.L + 1), coefj(Lv.L + 1), coefy(Lv.L + 1);
        cd il(1, 0);
        for (int n = 0; n <= Lv.L; ++n) {
            coef[n] = il * (2.0 * n + 1.0) * cd(jn[n], yn[n]);
            coefj[n] = il * (2.0 * n + 1.0) * jn[n];
            coefy[n] = il * (2.0 * n + 1.0) * yn[n];
            const cd hd = n == 0 ? -cd(jd[1], yd[1])
                                 : cd(jd[n - 1], yd[n - 1]) - (n + 1.0) / x * cd(jd[n], yd[n]);
            coefd[n] = il * (2.0 * n + 1.0) * rn * hd;
            il *= cd(0, 1);
        }
        for (int q = 0; q < Lv.K; ++q) {
            double kh[3];
            khat(Lv, q, kh);
            double c = (kh[0] * r[0] + kh[1] * r[1] + kh[2] * r[2]) / rn;
            cd s(0, 0), sd(0, 0), sj(0, 0), sy(0, 0);
            double p0 = 1.0, p1 = c;
            for (int n = 0; n <= Lv.L; ++n) {
                double pn;
                if (n == 0) pn = p0;
                else if (n == 1) pn = p1;
                else {
                    pn = ((2.0 * n - 1.0) * c * p1 - (n - 1.0) * p0) / n;
                    p0 = p1;
                    p1 = pn;
                }
                s += coef[n] * pn;
                sd += coefd[n] * pn;
                sj += coefj[n] * pn;
                sy += coefy[n] * pn;
            }
            Lv.alpha[(size_t)t * Lv.K + q] = s;
            Lv.alpha_dk[(size_t)t * Lv.K + q] = sd;
            Lv.alpha_j[(size_t)t * Lv.K + q] = sj;
            Lv.alpha_y[(size_t)t * Lv.K + q] = sy;
        }
    }
}

// Eq. (SinKer)'s table up to its factor -i: sum_{l=0}^{L} i^l (2l+1)
// j_l(k r) P_l(khat . rhat) for the sibling offsets of one level.
static void sibling_table(const Level &Lv, SibLevel &S, double k)
{
    S.alpha.assign((size_t)S.ntype * Lv.K, cd(0, 0));
    std::vector<double> jn;
    for (int t = 0; t < S.ntype; ++t) {
        double r[3] = {Lv.a * S.type_off[3 * t], Lv.a * S.type_off[3 * t + 1], Lv.a * S.type_off[3 * t + 2]};
        double rn = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        sph_bessel_j(Lv.L, k * rn, jn);
        std::vector<cd> coef(Lv.L + 1);
        cd il(1, 0);
        for (int n = 0; n <= Lv.L; ++n) {
            coef[n] = il * (2.0 * n + 1.0) * jn[n];
            il *= cd(0, 1);
        }
        for (int q = 0; q < Lv.K; ++q) {
            double kh[3];
            khat(Lv, q, kh);
            double c = (kh[0] * r[0] + kh[1] * r[1] + kh[2] * r[2]) / rn;
            cd s(0, 0);
            double p0 = 1.0, p1 = c;
            for (int n = 0; n <= Lv.L; ++n) {
                double pn;
                if (n == 0) pn = p0;
                else if (n == 1) pn = p1;
                else {
                    pn = ((2.0 * n - 1.0) * c * p1 - (n - 1.0) * p0) / n;
                    p0 = p1;
                    p1 = pn;
                }
                s += coef[n] * pn;
            }
            S.alpha[(size_t)t * Lv.K + q] = s;
        }
    }
}

// -------------------------------------------------------------- build ---
std::string build_plan_host(PlanHost &P, const double *verts, int64_t nv, const int32_t *tris,
                            int64_t nt, double k, int levels, double digits, int order, double eta)
{
    if (!verts || !tris || nv < 3 || nt < 1) return "mesh arrays missing or empty";
    if (!(k > 0) || !std::isfinite(k)) return "k must be positive and finite";
    if (levels < 2 || levels > 21) return "levels must be in 2..21";
    if (!(digits >= 1 && digits <= 15)) return "digits must be in 1..15";
    if (order < 4 || order > 12 || (order & 1)) return "interp_order must be even, 4..12";
    if (nt > (int64_t)1 << 30 || nv > (int64_t)1 << 30) return "mesh too large";
    P.k = k; P.digits = digits; P.levels = levels; P.leaf = levels - 1; P.order = order; P.eta = eta;
    P.V.assign(verts, verts + 3 * nv);
    P.T.assign(tris, tris + 3 * nt);
    for (int64_t i = 0; i < 3 * nv; ++i)
        if (!std::isfinite(P.V[i])) return "non-finite vertex coordinate";
    for (int64_t t = 0; t < nt; ++t) {
        const int32_t *x = &P.T[3 * t];
        for (int e = 0; e < 3; ++e)
            if (x[e] < 0 || x[e] >= nv) return "triangle vertex index out of range";
        if (x[0] == x[1] || x[1] == x[2] || x[0] == x[2]) return "degenerate triangle (repeated vertex)";
        const double *a = &P.V[3 * x[0]], *b = &P.V[3 * x[1]], *c = &P.V[3 * x[2]];
        double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, v[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
        double n[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
        if (!(n[0] * n[0] + n[1] * n[1] + n[2] * n[2] > 0)) return "degenerate triangle (zero area)";
    }

    // --- RWG list in canonical order
    struct HE { int32_t lo, hi, back, tri, opp; };
    std::vector<HE> he((size_t)3 * nt);
    for (int64_t t = 0; t < nt; ++t)
        for (int e = 0; e < 3; ++e) {
            int32_t a = P.T[3 * t + e], b = P.T[3 * t + (e + 1) % 3], c = P.T[3 * t + (e + 2) % 3];
            he[3 * t + e] = {std::min(a, b), std::max(a, b), a < b ? 0 : 1, (int32_t)t, c};
        }
    std::sort(he.begin(), he.end(), [](const HE &x, const HE &y) {
        if (x.lo != y.lo) return x.lo < y.lo;
        if (x.hi != y.hi) return x.hi < y.hi;
        return x.back < y.back;
    });
    for (size_t i = 0; i < he.size();) {
        size_t j = i;
        while (j < he.size() && he[j].lo == he[i].lo && he[j].hi == he[i].hi) ++j;
        if (j - i > 2) return "non-manifold edge (three or more triangles)";
        if (j - i == 2) {
            if (he[i].back == he[i + 1].back) return "inconsistent triangle orientation across an edge";
            P.rwg.edge_v.push_back(he[i].lo);
            P.rwg.edge_v.push_back(he[i].hi);
            P.rwg.tri.push_back(he[i].tri);
            P.rwg.tri.push_back(he[i + 1].tri);
            P.rwg.vfree.push_back(he[i].opp);
            P.rwg.vfree.push_back(he[i + 1].opp);
            const double *a = &P.V[3 * he[i].lo], *b = &P.V[3 * he[i].hi];
            P.rwg.len.push_back(std::sqrt((a[0] - b[0]) * (a[0] - b[0]) + (a[1] - b[1]) * (a[1] - b[1]) +
                                          (a[2] - b[2]) * (a[2] - b[2])));
        }
        i = j;
    }
    P.N = (int64_t)P.rwg.len.size();
    if (P.N == 0) return "mesh has no interior edge (no RWG function)";
    if (P.N > (int64_t)1 << 30) return "too many unknowns";

    // --- enclosing cube (level 0)
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t t = 0; t < 3 * nt; ++t) {
        const double *p = &P.V[3 * P.T[t]];
        for (int d = 0; d < 3; ++d) { lo[d] = std::min(lo[d], p[d]); hi[d] = std::max(hi[d], p[d]); }
    }
    P.root_side = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
    if (!(P.root_side > 0)) return "mesh has zero extent";
    for (int d = 0; d < 3; ++d) {
        P.root_center[d] = 0.5 * (lo[d] + hi[d]);
        P.origin[d] = P.root_center[d] - 0.5 * P.root_side;
    }
    P.lv.resize(levels);
    for (int l = 0; l < levels; ++l) {
        P.lv[l].l = l;
        P.lv[l].a = P.root_side / (double)((int64_t)1 << l);
    }

    // --- leaf boxes by edge midpoint, Morton order
    const int leaf = P.leaf;
    const int64_t nside = (int64_t)1 << leaf;
    const double aleaf = P.lv[leaf].a;
    std::vector<uint64_t> ucode(P.N);
    for (int64_t n = 0; n < P.N; ++n) {
        const double *a = &P.V[3 * P.rwg.edge_v[2 * n]], *b = &P.V[3 * P.rwg.edge_v[2 * n + 1]];
        int64_t ix[3];
        for (int d = 0; d < 3; ++d) {
            double m = 0.5 * (a[d] + b[d]);
            int64_t i = (int64_t)std::floor((m - P.origin[d]) / aleaf);
            ix[d] = std::max<int64_t>(0, std::min<int64_t>(nside - 1, i));
        }
        ucode[n] = morton(ix[0], ix[1], ix[2]);
    }
    P.perm.resize(P.N);
    std::iota(P.perm.begin(), P.perm.end(), 0);
    std::stable_sort(P.perm.begin(), P.perm.end(), [&](int64_t x, int64_t y) { return ucode[x] < ucode[y]; });
    {
        Level &Lf = P.lv[leaf];
        P.box_ptr.assign(1, 0);
        P.leaf_box.assign(P.N, -1);
        for (int64_t i = 0; i < P.N; ++i) {
            uint64_t c = ucode[P.perm[i]];
            if (Lf.code.empty() || Lf.code.back() != c) {
                if (!Lf.code.empty()) P.box_ptr.push_back((int32_t)i);
                Lf.code.push_back(c);
            }
            P.leaf_box[P.perm[i]] = (int32_t)Lf.code.size() - 1;
        }
        P.box_ptr.push_back((int32_t)P.N);
        P.max_leaf = 0;
        for (size_t b = 0; b + 1 < P.box_ptr.size(); ++b)
            P.max_leaf = std::max(P.max_leaf, P.box_ptr[b + 1] - P.box_ptr[b]);
    }
    // coarser levels, parents, children
    for (int l = leaf - 1; l >= 0; --l) {
        Level &C = P.lv[l + 1], &Pa = P.lv[l];
        Pa.code.clear();
        C.parent.assign(C.nbox(), 0);
        C.octant.assign(C.nbox(), 0);
        Pa.child_ptr.assign(1, 0);
        for (int b = 0; b < C.nbox(); ++b) {
            uint64_t pc = C.code[b] >> 3;
            if (Pa.code.empty() || Pa.code.back() != pc) {
                if (!Pa.code.empty()) Pa.child_ptr.push_back(b);
                Pa.code.push_back(pc);
            }
            C.parent[b] = (int32_t)Pa.code.size() - 1;
            C.octant[b] = (int32_t)(C.code[b] & 7);
        }
        Pa.child_ptr.push_back(C.nbox());
    }
    P.lv[0].parent.assign(P.lv[0].nbox(), -1);
    P.lv[0].octant.assign(P.lv[0].nbox(), 0);
    for (int l = 0; l < levels; ++l) {
        Level &Lv = P.lv[l];
        Lv.center.resize((size_t)3 * Lv.nbox());
        for (int b = 0; b < Lv.nbox(); ++b) {
            int64_t x, y, z;
            unmorton(Lv.code[b], x, y, z);
            Lv.center[3 * b] = P.origin[0] + (x + 0.5) * Lv.a;
            Lv.center[3 * b + 1] = P.origin[1] + (y + 0.5) * Lv.a;
            Lv.center[3 * b + 2] = P.origin[2] + (z + 0.5) * Lv.a;
        }
    }

    // per-level lookup code -> box
    std::vector<std::unordered_map<uint64_t, int>> lookup(levels);
    for (int l = 0; l < levels; ++l) {
        lookup[l].reserve(P.lv[l].nbox() * 2);
        for (int b = 0; b < P.lv[l].nbox(); ++b) lookup[l][P.lv[l].code[b]] = b;
    }
    auto neighbours = [&](int l, int b, std::vector<int> &out) {
        out.clear();
        int64_t x, y, z;
        unmorton(P.lv[l].code[b], x, y, z);
        const int64_t ns = (int64_t)1 << l;
        for (int dx = -1; dx <= 1; ++dx)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dz = -1; dz <= 1; ++dz) {
                    int64_t X = x + dx, Y = y + dy, Z = z + dz;
                    if (X < 0 || Y < 0 || Z < 0 || X >= ns || Y >= ns || Z >= ns) continue;
                    auto it = lookup[l].find(morton(X, Y, Z));
                    if (it != lookup[l].end()) out.push_back(it->second);
                }
        std::sort(out.begin(), out.end());
    };

    // --- near strips on the leaf level (B_m: the leaf box and its neighbours)
    {
        const Level &Lf = P.lv[leaf];
        std::vector<int> nb;
        P.nb_ptr.assign(1, 0);
        P.strip_off.assign(1, 0);
        P.col_ptr.assign(1, 0);
        for (int b = 0; b < Lf.nbox(); ++b) {
            neighbours(leaf, b, nb);
            int64_t ncols = 0;
            for (int c : nb) {
                P.nb_box.push_back(c);
                for (int32_t u = P.box_ptr[c]; u < P.box_ptr[c + 1]; ++u) P.strip_col.push_back(u);
                ncols += P.box_ptr[c + 1] - P.box_ptr[c];
            }
            P.nb_ptr.push_back((int32_t)P.nb_box.size());
            P.col_ptr.push_back((int32_t)P.strip_col.size());
            P.strip_off.push_back(P.strip_off.back() + ncols * (P.box_ptr[b + 1] - P.box_ptr[b]));
        }
        P.nnz = P.strip_off.back();
        if (P.strip_col.size() > (size_t)INT32_MAX) return "near structure too large";
        P.self_off.assign(1, 0);
        P.self_col_ptr.assign(1, 0);
        P.self_col.clear();
        for (int b = 0; b < Lf.nbox(); ++b) {
            const int64_t nr = P.box_ptr[b + 1] - P.box_ptr[b];
            for (int32_t u = P.box_ptr[b]; u < P.box_ptr[b + 1]; ++u) P.self_col.push_back(u);
            P.self_col_ptr.push_back((int32_t)P.self_col.size());
            P.self_off.push_back(P.self_off.back() + nr * nr);
        }
        P.self_nnz = P.self_off.back();
    }

    // --- sibling translations (sin-kernel product): level 1 .. leaf
    P.sib.assign(levels, SibLevel());
    if (leaf >= 1) make_grid(P.lv[1], k, digits);
    for (int l = 1; l <= leaf; ++l) {
        const Level &Lv = P.lv[l], &Pa = P.lv[l - 1];
        SibLevel &S = P.sib[l];
        std::vector<int> type_of(27, -1);
        S.grp_ptr.assign(1, 0);
        for (int pb = 0; pb < Pa.nbox(); ++pb) {
            const int c0 = Pa.child_ptr[pb], nc = Pa.child_ptr[pb + 1] - c0;
            for (int s = c0; s < c0 + nc; ++s) {
                int64_t X, Y, Z;
                unmorton(Lv.code[s], X, Y, Z);
                int16_t ty[8];
                for (int c = 0; c < 8; ++c) ty[c] = -1;
                for (int c = 0; c < nc; ++c) {
                    if (c0 + c == s) continue;
                    int64_t x, y, z;
                    unmorton(Lv.code[c0 + c], x, y, z);
                    const int dx = (int)(x - X), dy = (int)(y - Y), dz = (int)(z - Z);   // r_m - r_m'
                    const int key = (dx + 1) * 9 + (dy + 1) * 3 + (dz + 1);
                    if (type_of[key] < 0) {
                        type_of[key] = S.ntype++;
                        S.type_off.push_back(dx);
                        S.type_off.push_back(dy);
                        S.type_off.push_back(dz);
                    }
                    ty[c] = (int16_t)type_of[key];
                }
                S.grp_src.push_back(s);
                for (int c = 0; c < 8; ++c) S.grp_ty.push_back(ty[c]);
            }
            S.grp_ptr.push_back((int32_t)S.grp_src.size());
            S.max_grp = std::max(S.max_grp, nc);
        }
    }

    // --- far levels: grids, interaction lists, translation tables
    std::vector<int> nbp, nbs;
    for (int l = 2; l <= leaf; ++l) {
        Level &Lv = P.lv[l];
        make_grid(Lv, k, digits);
        std::vector<int> type_of(343, -1);
        Lv.il_ptr.assign(1, 0);
        Lv.il_src.clear();
        Lv.il_type.clear();
        Lv.type_off.clear();
        Lv.ntype = 0;
        for (int b = 0; b < Lv.nbox(); ++b) {
            int64_t x, y, z;
            unmorton(Lv.code[b], x, y, z);
            neighbours(l - 1, Lv.parent[b], nbp);
            for (int pn : nbp)
                for (int c = P.lv[l - 1].child_ptr[pn]; c < P.lv[l - 1].child_ptr[pn + 1]; ++c) {
                    int64_t X, Y, Z;
                    unmorton(Lv.code[c], X, Y, Z);
                    int dx = (int)(x - X), dy = (int)(y - Y), dz = (int)(z - Z);  // r_m - r_m'
                    if (std::abs(dx) <= 1 && std::abs(dy) <= 1 && std::abs(dz) <= 1) continue;
                    int key = (dx + 3) * 49 + (dy + 3) * 7 + (dz + 3);
                    if (type_of[key] < 0) {
                        type_of[key] = Lv.ntype++;
                        Lv.type_off.push_back(dx);
                        Lv.type_off.push_back(dy);
                        Lv.type_off.push_back(dz);
                    }
                    Lv.il_src.push_back(c);
                    Lv.il_type.push_back(type_of[key]);
                }
            Lv.il_ptr.push_back((int32_t)Lv.il_src.size());
            // at most 6^3 - 3^3 = 189 boxes: children of the parent's
            // neighbours that are not neighbours themselves
            if (Lv.il_ptr[b + 1] - Lv.il_ptr[b] > 189) return "interaction list longer than 189 (internal error)";
        }
        // grouped form: sources shared by the children of one parent
        {
            const Level &Pa = P.lv[l - 1];
            Lv.grp_ptr.assign(1, 0);
            Lv.grp_src.clear();
            Lv.grp_ty.clear();
            Lv.max_grp = 0;
            for (int pb = 0; pb < Pa.nbox(); ++pb) {
                const int c0 = Pa.child_ptr[pb], nc = Pa.child_ptr[pb + 1] - c0;
                neighbours(l - 1, pb, nbp);
                for (int pn : nbp)
                    for (int s = Pa.child_ptr[pn]; s < Pa.child_ptr[pn + 1]; ++s) {
                        int64_t X, Y, Z;
                        unmorton(Lv.code[s], X, Y, Z);
                        int16_t ty[8];
                        bool any = false;
                        for (int c = 0; c < 8; ++c) {
                            ty[c] = -1;
                            if (c >= nc) continue;
                            int64_t x, y, z;
                            unmorton(Lv.code[c0 + c], x, y, z);
                            int dx = (int)(x - X), dy = (int)(y - Y), dz = (int)(z - Z);
                            if (std::abs(dx) <= 1 && std::abs(dy) <= 1 && std::abs(dz) <= 1) continue;
                            int t = type_of[(dx + 3) * 49 + (dy + 3) * 7 + (dz + 3)];
                            if (t < 0) return "grouped interaction list disagrees with the per-box list";
                            ty[c] = (int16_t)t;
                            any = true;
                        }
                        if (!any) continue;
                        Lv.grp_src.push_back(s);
                        for (int c = 0; c < 8; ++c) Lv.grp_ty.push_back(ty[c]);
                    }
                Lv.grp_ptr.push_back((int32_t)Lv.grp_src.size());
                Lv.max_grp = std::max(Lv.max_grp, Lv.grp_ptr[pb + 1] - Lv.grp_ptr[pb]);
            }
            if (Lv.max_grp > 216) return "grouped source list longer than 216 (internal error)";
            // distinct types per parent and the entries' local type indices
            Lv.lty_ptr.assign(1, 0);
            Lv.lty.clear();
            Lv.grp_lty.assign(Lv.grp_ty.size(), (int16_t)-1);
            Lv.max_lty = 0;
            std::vector<int> local(Lv.ntype, -1);
            for (int pb = 0; pb + 1 < (int)Lv.grp_ptr.size(); ++pb) {
                const int base = (int)Lv.lty.size();
                for (int e = Lv.grp_ptr[pb]; e < Lv.grp_ptr[pb + 1]; ++e)
                    for (int c = 0; c < 8; ++c) {
                        const int ty = Lv.grp_ty[(size_t)e * 8 + c];
                        if (ty < 0) continue;
                        if (local[ty] < 0) {
                            local[ty] = (int)Lv.lty.size() - base;
                            Lv.lty.push_back(ty);
                        }
                        Lv.grp_lty[(size_t)e * 8 + c] = (int16_t)local[ty];
                    }
                for (size_t i = base; i < Lv.lty.size(); ++i) local[Lv.lty[i]] = -1;
                Lv.lty_ptr.push_back((int32_t)Lv.lty.size());
                Lv.max_lty = std::max(Lv.max_lty, (int)Lv.lty.size() - base);
            }
        }
        translation_table(Lv, k);
    }

    for (int l = 1; l <= leaf; ++l) sibling_table(P.lv[l], P.sib[l], k);

    // --- interpolation (child l+1 -> parent l) and phase shifts, 1 <= l < leaf
    // (level 1 serves the sibling scheme only)
    for (int l = 1; l < leaf; ++l) {
        Level &Pa = P.lv[l];
        const Level &C = P.lv[l + 1];
        theta_stencil(C.th, Pa.th, order, Pa.th_up);
        phi_stencil(C.nph, Pa.ph, order, Pa.ph_up);
        // anterpolation = W_child^-1 * Interp^T * W_parent (separable weights)
        const double phr = (double)C.nph / (double)Pa.nph;
        transpose_stencil(Pa.ph_up, C.nph, [&](int, int) { return phr; }, Pa.ph_dn);
        transpose_stencil(Pa.th_up, C.nth, [&](int t, int j) { return Pa.wt[t] / C.wt[j]; }, Pa.th_dn);
        win_stencil(Pa.th_up, C.nth, true, kWinMax, Pa.wu_th);
        win_stencil(Pa.ph_up, C.nph, false, kWinMax, Pa.wu_ph);
        win_stencil(Pa.ph_dn, Pa.nph, false, kWinMax, Pa.wd_ph);
        win_stencil(Pa.th_dn, Pa.nth, true, kWinMax, Pa.wd_th);
        Pa.shift.resize((size_t)8 * Pa.K);
        Pa.shift_dk.resize((size_t)8 * Pa.K);
        Pa.shift_xy.resize((size_t)8 * Pa.K);
        Pa.gam.resize((size_t)8 * Pa.nth);
        for (int o = 0; o < 8; ++o) {
            const double h = 0.5 * C.a;
            double d[3] = {-h * (((o >> 2) & 1) ? 1 : -1), -h * (((o >> 1) & 1) ? 1 : -1), -h * ((o & 1) ? 1 : -1)};
            for (int q = 0; q < Pa.K; ++q) {
                double kh[3];
                khat(Pa, q, kh);
                const double kd = kh[0] * d[0] + kh[1] * d[1] + kh[2] * d[2];
                double ph = k * kd;
                Pa.shift[(size_t)o * Pa.K + q] = cd(std::cos(ph), std::sin(ph));
                Pa.shift_dk[(size_t)o * Pa.K + q] = cd(0.0, kd) * cd(std::cos(ph), std::sin(ph));
                const double pxy = k * (kh[0] * d[0] + kh[1] * d[1]);
                Pa.shift_xy[(size_t)o * Pa.K + q] = cd(std::cos(pxy), std::sin(pxy));
            }
            for (int t = 0; t < Pa.nth; ++t) {
                const double pz = k * Pa.ct[t] * d[2];
                Pa.gam[(size_t)o * Pa.nth + t] = cd(std::cos(pz), std::sin(pz));
            }
        }
    }
    return "";
}

}  // namespace mlfma
