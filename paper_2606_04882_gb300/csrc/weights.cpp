// Host FP64 stencil geometry, weight schemes and stability bound
// (fd_weights, fd_cfl_limit, fd_ricker).
//
// Geometry: Section 4.1 (shapes through Q, P0(q), P(q)); 3D = union of the 2D
// shape in the three coordinate planes.  Unknowns are one weight per symmetry
// orbit (sorted absolute offsets), each equation carrying the orbit's sum over
// its offsets - the reading of the symmetric c_{p,q} = a_{p,q} + a_{q,p}
// passage of Section 4.1.
//
// Solvers: the Taylor cross uses the closed form of the centred second
// derivative; moment systems (SpecTE-theta, DispTE, DispTE-theta) are solved
// by Gaussian elimination in double-double arithmetic (portable, deterministic
// on every host); least-squares schemes assemble the quadrature design matrix
// and take the truncated minimum-norm solution from a one-sided Jacobi SVD.
#include <algorithm>
#include <functional>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "internal.h"
#include "runtime.h"

namespace fdw {

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kLsRcond = 1e-10;   // relative singular-value cutoff of the LS schemes

// ------------------------------- geometry ---------------------------------

using Off = std::array<int, 3>;   // (dz, dy, dx); 2D uses (dz, 0, dx)

bool offaxis(int shape, int M, int N, int q, int &p0, int &p1)
{
    switch (shape) {
    case FD_CROSS: return false;
    case FD_RHOMBUS: if (q > M / 2) return false; p0 = q; p1 = M - q; return true;
    case FD_CROSS_RHOMBUS: if (q > N / 2) return false; p0 = q; p1 = N - q; return true;
    case FD_SQUARE: if (q > M) return false; p0 = q; p1 = M; return true;
    case FD_CROSS_SQUARE: if (q > N) return false; p0 = q; p1 = M; return true;
    }
    return false;
}

std::vector<std::array<int, 2>> points2d(int shape, int M, int N)
{
    std::vector<std::array<int, 2>> pts;
    auto add = [&](int a, int b) {
        for (auto &t : pts)
            if (t[0] == a && t[1] == b) return;
        pts.push_back({a, b});
    };
    add(0, 0);
    for (int m = 1; m <= M; ++m) { add(m, 0); add(-m, 0); add(0, m); add(0, -m); }
    for (int q = 1; q <= M; ++q) {
        int p0, p1;
        if (!offaxis(shape, M, N, q, p0, p1)) continue;
        for (int p = p0; p <= p1; ++p)
            for (int sp = -1; sp <= 1; sp += 2)
                for (int sq = -1; sq <= 1; sq += 2) { add(sp * p, sq * q); add(sq * q, sp * p); }
    }
    return pts;
}

struct Orbit {
    std::array<int, 3> key;         // sorted |offsets|, descending
    std::vector<Off> offs;
};

std::vector<Orbit> build_orbits(int dim, int shape, int M, int N)
{
    std::vector<Off> offs;
    for (auto &t : points2d(shape, M, N)) {
        if (dim == 2) {
            offs.push_back({t[1], 0, t[0]});
        } else {
            Off cand[3] = {{0, t[1], t[0]}, {t[1], 0, t[0]}, {t[1], t[0], 0}};
            for (auto &c : cand)
                if (std::find(offs.begin(), offs.end(), c) == offs.end()) offs.push_back(c);
        }
    }
    std::map<std::array<int, 3>, Orbit> m;
    for (auto &o : offs) {
        std::array<int, 3> k = {std::abs(o[0]), std::abs(o[1]), std::abs(o[2])};
        std::sort(k.begin(), k.end(), [](int a, int b) { return a > b; });
        auto &orb = m[k];
        orb.key = k;
        orb.offs.push_back(o);
    }
    std::vector<Orbit> out;
    for (auto &kv : m) out.push_back(kv.second);
    std::sort(out.begin(), out.end(), [](const Orbit &a, const Orbit &b) {
        return a.key < b.key;   // centre (0,0,0) first
    });
    return out;
}

// ------------------------------ double-double -----------------------------

struct dd {
    double hi, lo;
};
inline dd two_sum(double a, double b)
{
    double s = a + b, bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
inline dd dd_add(dd a, dd b)
{
    dd s = two_sum(a.hi, b.hi);
    dd t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return two_sum(s.hi, s.lo);
}
inline dd dd_neg(dd a) { return {-a.hi, -a.lo}; }
inline dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }
inline dd dd_mul(dd a, dd b)
{
    double p = a.hi * b.hi;
    double e = std::fma(a.hi, b.hi, -p);
    e += a.hi * b.lo + a.lo * b.hi;
    return two_sum(p, e);
}
inline dd dd_div(dd a, dd b)
{
    double q1 = a.hi / b.hi;
    dd r = dd_sub(a, dd_mul({q1, 0.0}, b));
    double q2 = r.hi / b.hi;
    r = dd_sub(r, dd_mul({q2, 0.0}, b));
    double q3 = r.hi / b.hi;
    dd q = two_sum(q1, q2);
    return dd_add(q, {q3, 0.0});
}
inline dd D(double x) { return {x, 0.0}; }

using Mat = std::vector<std::vector<dd>>;

// Solve the square system A x = b (Gaussian elimination, partial pivoting).
bool dd_solve(Mat A, std::vector<dd> b, std::vector<dd> &x)
{
    const int n = (int)A.size();
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(A[r][c].hi) > std::fabs(A[piv][c].hi)) piv = r;
        if (A[piv][c].hi == 0.0) return false;
        std::swap(A[c], A[piv]);
        std::swap(b[c], b[piv]);
        for (int r = c + 1; r < n; ++r) {
            dd f = dd_div(A[r][c], A[c][c]);
            if (f.hi == 0.0) continue;
            for (int k = c; k < n; ++k) A[r][k] = dd_sub(A[r][k], dd_mul(f, A[c][k]));
            b[r] = dd_sub(b[r], dd_mul(f, b[c]));
        }
    }
    x.assign(n, D(0.0));
    for (int r = n - 1; r >= 0; --r) {
        dd s = b[r];
        for (int k = r + 1; k < n; ++k) s = dd_sub(s, dd_mul(A[r][k], x[k]));
        x[r] = dd_div(s, A[r][r]);
    }
    return true;
}

// Indices of a maximal set of independent rows (elimination with a relative
// threshold far below double-double resolution of the integer-like systems).
std::vector<int> independent_rows(const Mat &A)
{
    std::vector<int> keep;
    std::vector<std::vector<dd>> basis;
    std::vector<int> pivc;
    double scale = 0.0;
    for (auto &r : A)
        for (auto &v : r) scale = std::max(scale, std::fabs(v.hi));
    for (size_t i = 0; i < A.size(); ++i) {
        std::vector<dd> v = A[i];
        for (size_t b = 0; b < basis.size(); ++b) {
            const int pc = pivc[b];
            if (v[pc].hi == 0.0) continue;
            dd f = dd_div(v[pc], basis[b][pc]);
            for (size_t k = 0; k < v.size(); ++k) v[k] = dd_sub(v[k], dd_mul(f, basis[b][k]));
        }
        int pc = -1;
        double best = 0.0;
        for (size_t k = 0; k < v.size(); ++k)
            if (std::fabs(v[k].hi) > best) { best = std::fabs(v[k].hi); pc = (int)k; }
        if (pc >= 0 && best > 1e-24 * std::max(scale, 1.0)) {
            basis.push_back(v);
            pivc.push_back(pc);
            keep.push_back((int)i);
        }
    }
    return keep;
}

// Minimum-norm least-squares solution: full column rank -> normal equations
// over all rows; otherwise x = A_r^T (A_r A_r^T)^{-1} b_r on independent rows.
bool dd_lstsq(const Mat &A, const std::vector<dd> &b, std::vector<double> &x)
{
    const int n = (int)A[0].size();
    std::vector<int> rows = independent_rows(A);
    std::vector<dd> sol;
    if ((int)rows.size() == n) {
        Mat N(n, std::vector<dd>(n, D(0.0)));
        std::vector<dd> r(n, D(0.0));
        for (int i = 0; i < n; ++i) {
            for (int j = 0; j < n; ++j)
                for (size_t k = 0; k < A.size(); ++k) N[i][j] = dd_add(N[i][j], dd_mul(A[k][i], A[k][j]));
            for (size_t k = 0; k < A.size(); ++k) r[i] = dd_add(r[i], dd_mul(A[k][i], b[k]));
        }
        if (!dd_solve(N, r, sol)) return false;
    } else {
        const int m = (int)rows.size();
        Mat G(m, std::vector<dd>(m, D(0.0)));
        std::vector<dd> br(m);
        for (int i = 0; i < m; ++i) {
            br[i] = b[rows[i]];
            for (int j = 0; j < m; ++j)
                for (int k = 0; k < n; ++k)
                    G[i][j] = dd_add(G[i][j], dd_mul(A[rows[i]][k], A[rows[j]][k]));
        }
        std::vector<dd> y;
        if (!dd_solve(G, br, y)) return false;
        sol.assign(n, D(0.0));
        for (int k = 0; k < n; ++k)
            for (int i = 0; i < m; ++i) sol[k] = dd_add(sol[k], dd_mul(A[rows[i]][k], y[i]));
    }
    x.resize(n);
    for (int i = 0; i < n; ++i) x[i] = sol[i].hi + sol[i].lo;
    return true;
}

dd dd_pow(dd a, int e)
{
    dd r = D(1.0);
    for (int i = 0; i < e; ++i) r = dd_mul(r, a);
    return r;
}

double factorial(int n)
{
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

// ----------------------------- moment systems -----------------------------

// Mixed-derivative equations kept up to order r: N for cross-rhombus (square
// system, as Section 4.2 states), none for the cross, all for the others.
int mixed_order(int shape, int M, int N)
{
    if (shape == FD_CROSS) return 1;
    if (shape == FD_CROSS_RHOMBUS) return std::max(1, N);
    return M;
}

// DispTE (C > 0) / spatial Taylor (C = 0) moment equations: for exponent
// tuples e (sum r) sum_orb a sum_{o in orb} prod o_i^(2 e_i) = 2 C^(2r-2)
// r!/prod e_i! / ((2r)!/prod (2e_i)!), r = 0 -> 0.
void moment_system(int dim, const std::vector<Orbit> &orbs, int M, double C, int rmix, Mat &A,
                   std::vector<dd> &b)
{
    A.clear();
    b.clear();
    const dd Cd = D(C);
    for (int r = 0; r <= M; ++r) {
        for (int e0 = r; e0 >= 0; --e0)
            for (int e1 = std::min(e0, r - e0); e1 >= 0; --e1) {
                int e2 = r - e0 - e1;
                if (dim == 2 && e2 != 0) continue;
                if (e2 > e1) continue;
                const int e[3] = {e0, e1, dim == 3 ? e2 : 0};
                if (dim == 2 && e1 + e0 != r) continue;
                const int nnz = (e[0] > 0) + (e[1] > 0) + (e[2] > 0);
                if (nnz >= 2 && r > rmix) continue;
                std::vector<dd> row;
                for (auto &orb : orbs) {
                    double s = 0.0;   // integer-valued, exact in double for M <= 16
                    for (auto &o : orb.offs) {
                        // exponents apply to the (sorted) axes of the tuple:
                        // sum over the orbit is symmetric, so any axis order works
                        const int c[3] = {o[2], dim == 3 ? o[1] : o[0], dim == 3 ? o[0] : 0};
                        double t = 1.0;
                        for (int i = 0; i < 3; ++i)
                            for (int k = 0; k < 2 * e[i]; ++k) t *= c[i];
                        s += t;
                    }
                    row.push_back(D(s));
                }
                A.push_back(row);
                if (r == 0) {
                    b.push_back(D(0.0));
                } else {
                    double mn = factorial(r), mn2 = factorial(2 * r);
                    for (int i = 0; i < 3; ++i) { mn /= factorial(e[i]); mn2 /= factorial(2 * e[i]); }
                    dd cp = r == 1 ? D(1.0) : dd_pow(Cd, 2 * r - 2);
                    b.push_back(dd_div(dd_mul(dd_mul(D(2.0), cp), D(mn)), D(mn2)));
                }
            }
    }
}

// Polar (theta) system at one angle: r = 0: sum mult a = 0; r >= 1:
// sum_orb a sum_o (o . khat)^(2r) = 2 C^(2r-2), khat = (cos theta, sin theta)
// acting on (dx, dz).
void theta_system(const std::vector<Orbit> &orbs, int M, double C, double theta, Mat &A,
                  std::vector<dd> &b)
{
    A.clear();
    b.clear();
    std::vector<dd> r0;
    for (auto &orb : orbs) r0.push_back(D((double)orb.offs.size()));
    A.push_back(r0);
    b.push_back(D(0.0));
    const double cx = std::cos(theta), cz = std::sin(theta);
    for (int r = 1; r <= M; ++r) {
        std::vector<dd> row;
        for (auto &orb : orbs) {
            dd s = D(0.0);
            for (auto &o : orb.offs) {
                dd pr = dd_add(dd_mul(D((double)o[2]), D(cx)), dd_mul(D((double)o[0]), D(cz)));
                s = dd_add(s, dd_pow(pr, 2 * r));
            }
            row.push_back(s);
        }
        A.push_back(row);
        b.push_back(dd_mul(D(2.0), r == 1 ? D(1.0) : dd_pow(D(C), 2 * r - 2)));
    }
}

// --------------------------- least-squares schemes ------------------------

void gauss_legendre(int n, double a, double b, std::vector<double> &x, std::vector<double> &w)
{
    x.resize(n);
    w.resize(n);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5)), pp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p1 = 1.0, p2 = 0.0;
            for (int j = 1; j <= n; ++j) {
                double p3 = p2;
                p2 = p1;
                p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
            }
            pp = n * (z * p1 - p2) / (z * z - 1.0);
            double z1 = z;
            z = z1 - p1 / pp;
            if (std::fabs(z - z1) < 1e-15) break;
        }
        x[i] = 0.5 * (a + b) - 0.5 * (b - a) * z;
        w[i] = (b - a) / ((1.0 - z * z) * pp * pp);
    }
}

double taylor_cos(double x, int M)
{
    double term = 1.0, s = 1.0;
    for (int r = 1; r <= M; ++r) {
        term *= -x * x / ((2.0 * r - 1.0) * (2.0 * r));
        s += term;
    }
    return s;
}

// One-sided Jacobi SVD of A (m x n, column-major in `a`): rotates the columns
// until they are mutually orthogonal, so that afterwards column j of `a` is
// sigma_j u_j and A V = U Sigma with V (n x n, column-major) the rotations.
void jacobi_orthogonalise(std::vector<double> &a, int m, int n, std::vector<double> &V)
{
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    auto col = [&](int j) { return &a[(size_t)j * m]; };
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double al = 0, be = 0, ga = 0;
                const double *ap = col(p), *aq = col(q);
                for (int i = 0; i < m; ++i) { al += ap[i] * ap[i]; be += aq[i] * aq[i]; ga += ap[i] * aq[i]; }
                if (al == 0.0 || be == 0.0) continue;
                const double c0 = std::fabs(ga) / std::sqrt(al * be);
                off = std::max(off, c0);
                if (c0 < 1e-15) continue;
                const double zeta = (be - al) / (2.0 * ga);
                const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / std::sqrt(1.0 + t * t), s = c * t;
                double *xp = col(p), *xq = col(q);
                for (int i = 0; i < m; ++i) {
                    const double u = xp[i], v = xq[i];
                    xp[i] = c * u - s * v;
                    xq[i] = s * u + c * v;
                }
                for (int i = 0; i < n; ++i) {
                    const double u = V[(size_t)p * n + i], v = V[(size_t)q * n + i];
                    V[(size_t)p * n + i] = c * u - s * v;
                    V[(size_t)q * n + i] = s * u + c * v;
                }
            }
        if (off < 1e-15) break;
    }
}

std::vector<double> column_norms(const std::vector<double> &a, int m, int n)
{
    std::vector<double> sig(n);
    for (int j = 0; j < n; ++j) {
        double s = 0.0;
        for (int i = 0; i < m; ++i) s += a[(size_t)j * m + i] * a[(size_t)j * m + i];
        sig[j] = std::sqrt(s);
    }
    return sig;
}

// Minimum-norm least squares through the SVD: x = V Sigma^+ U^T b, singular
// values at or below rcond * sigma_max dropped.
bool jacobi_lstsq(std::vector<double> a, int m, int n, const std::vector<double> &b,
                  double rcond, std::vector<double> &x)
{
    std::vector<double> V;
    jacobi_orthogonalise(a, m, n, V);
    const std::vector<double> sig = column_norms(a, m, n);
    const double smax = *std::max_element(sig.begin(), sig.end());
    if (smax == 0.0) return false;
    x.assign(n, 0.0);
    for (int j = 0; j < n; ++j) {
        if (sig[j] <= rcond * smax) continue;
        double utb = 0.0;
        for (int i = 0; i < m; ++i) utb += a[(size_t)j * m + i] * b[i];
        const double coef = utb / (sig[j] * sig[j]);   // u_j = col_j / sigma_j
        for (int k = 0; k < n; ++k) x[k] += V[(size_t)j * n + k] * coef;
    }
    return true;
}

// Weighted design matrix of the LS schemes (column-major, m rows), its
// right-hand side and the orbits of its columns (every non-centre orbit).
void ls_design(int dim, const std::vector<Orbit> &orbs, int M, int scheme, int basis, double C,
               double band, std::vector<double> &A, int &m, int &n, std::vector<double> &rhs,
               std::vector<int> &cols)
{
    if (basis == FD_LS_PAPER) basis = scheme == FD_SPECLS ? FD_LS_TAYLOR : FD_LS_COSINE;
    const double b = band > 0 ? band : kPi / 2;
    std::vector<double> xb, wb;
    gauss_legendre(64, 0.0, b, xb, wb);
    // directions folded by the stencil's symmetry group: 2D theta in [0, pi/4]
    // (x8); 3D the octant x,y,z >= 0 (x8)
    std::vector<std::array<double, 3>> dirs;   // (kz, ky, kx)
    std::vector<double> dw;
    if (dim == 2) {
        std::vector<double> th, wt;
        gauss_legendre(48, 0.0, kPi / 4, th, wt);
        for (size_t i = 0; i < th.size(); ++i) {
            dirs.push_back({std::sin(th[i]), 0.0, std::cos(th[i])});
            dw.push_back(8.0 * wt[i]);
        }
    } else {
        std::vector<double> mu, wm, ph, wp;
        gauss_legendre(32, 0.0, 1.0, mu, wm);
        gauss_legendre(32, 0.0, kPi / 2, ph, wp);
        for (size_t i = 0; i < mu.size(); ++i)
            for (size_t j = 0; j < ph.size(); ++j) {
                const double st = std::sqrt(1.0 - mu[i] * mu[i]);
                dirs.push_back({mu[i], st * std::sin(ph[j]), st * std::cos(ph[j])});
                dw.push_back(8.0 * wm[i] * wp[j]);
            }
    }
    cols.clear();
    for (size_t k = 0; k < orbs.size(); ++k)
        if (orbs[k].key[0] || orbs[k].key[1] || orbs[k].key[2]) cols.push_back((int)k);
    n = (int)cols.size();
    m = (int)(xb.size() * dirs.size());
    A.assign((size_t)m * n, 0.0);
    rhs.assign(m, 0.0);
    int row = 0;
    for (size_t ib = 0; ib < xb.size(); ++ib)
        for (size_t id = 0; id < dirs.size(); ++id, ++row) {
            const double beta = xb[ib];
            const double sw = std::sqrt(wb[ib] * dw[id]);
            double target;
            if (scheme == FD_SPECLS) target = beta * beta;
            else target = C > 0 ? (2.0 - 2.0 * std::cos(C * beta)) / (C * C) : beta * beta;
            for (int c = 0; c < n; ++c) {
                double s = 0.0;
                for (auto &o : orbs[cols[c]].offs) {
                    const double proj = beta * (dirs[id][0] * o[0] + dirs[id][1] * o[1] + dirs[id][2] * o[2]);
                    s += 1.0 - (basis == FD_LS_TAYLOR ? taylor_cos(proj, M) : std::cos(proj));
                }
                if (basis == FD_LS_COSINE) s /= target;
                A[(size_t)c * m + row] = s * sw;
            }
            rhs[row] = (basis == FD_LS_COSINE ? 1.0 : target) * sw;
        }
}

int ls_weights(int dim, const std::vector<Orbit> &orbs, int M, int scheme, int basis, double C,
               double band, std::vector<double> &w)
{
    std::vector<double> A, rhs;
    std::vector<int> cols;
    int m = 0, n = 0;
    ls_design(dim, orbs, M, scheme, basis, C, band, A, m, n, rhs, cols);
    std::vector<double> x;
    if (!jacobi_lstsq(A, m, n, rhs, kLsRcond, x)) return FD_ERR_SINGULAR;
    w.assign(orbs.size(), 0.0);
    double centre = 0.0;
    for (int c = 0; c < n; ++c) {
        w[cols[c]] = x[c];
        centre -= (double)orbs[cols[c]].offs.size() * x[c];
    }
    w[0] = centre;
    return FD_OK;
}

// ------------------------------ dispatcher --------------------------------

int check_desc(const fd_stencil_desc *d)
{
    if (!d) return set_error(FD_ERR_ARG, "stencil descriptor is NULL");
    if (d->dim != 2 && d->dim != 3) return set_error(FD_ERR_ARG, "dim must be 2 or 3 (got %d)", d->dim);
    if (d->M < 1 || d->M > kMaxM) return set_error(FD_ERR_ARG, "radius M must be in [1, %d] (got %d)", kMaxM, d->M);
    if (d->shape < FD_CROSS || d->shape > FD_SQUARE) return set_error(FD_ERR_ARG, "unknown shape %d", d->shape);
    if (d->scheme < FD_SPATTE || d->scheme > FD_DISPLS) return set_error(FD_ERR_ARG, "unknown scheme %d", d->scheme);
    if (d->shape == FD_CROSS_RHOMBUS && (d->N < 1 || d->N > d->M))
        return set_error(FD_ERR_ARG, "cross-rhombus needs 1 <= N <= M (got N=%d)", d->N);
    if (d->shape == FD_CROSS_SQUARE && (d->N < 0 || d->N > d->M))
        return set_error(FD_ERR_ARG, "cross-square needs 0 <= N <= M (got N=%d)", d->N);
    if ((d->scheme == FD_DISPTE || d->scheme == FD_DISPLS || d->scheme == FD_DISPTE_THETA) &&
        !(d->courant >= 0.0 && d->courant < 10.0))
        return set_error(FD_ERR_ARG, "courant number must be in [0, 10) (got %g)", d->courant);
    if (d->ls_basis < FD_LS_PAPER || d->ls_basis > FD_LS_COSINE)
        return set_error(FD_ERR_ARG, "unknown ls_basis %d", d->ls_basis);
    return FD_OK;
}

}  // namespace

int compute_weights(const fd_stencil_desc *d, std::vector<std::array<int, 3>> &keys,
                    std::vector<int> &mult, std::vector<double> &w,
                    std::vector<std::array<int, 3>> *offsets, std::vector<int> *off_orbit)
{
    int st = check_desc(d);
    if (st) return st;
    const int dim = d->dim, M = d->M, N = d->N, shape = d->shape;
    auto orbs = build_orbits(dim, shape, M, N);
    keys.clear();
    mult.clear();
    for (auto &o : orbs) {
        keys.push_back(o.key);
        mult.push_back((int)o.offs.size());
    }
    if (offsets) {
        offsets->clear();
        off_orbit->clear();
        for (size_t k = 0; k < orbs.size(); ++k)
            for (auto &o : orbs[k].offs) { offsets->push_back(o); off_orbit->push_back((int)k); }
    }
    w.assign(orbs.size(), 0.0);
    auto is_axis = [](const std::array<int, 3> &k) { return k[1] == 0; };
    if (d->scheme == FD_SPATTE) {
        // a_m = 2 (-1)^(m+1) (M!)^2 / (m^2 (M-m)! (M+m)!), centre -2 dim sum a_m
        double centre = 0.0;
        for (size_t k = 0; k < orbs.size(); ++k) {
            if (!is_axis(orbs[k].key) || orbs[k].key[0] == 0) continue;
            const int m = orbs[k].key[0];
            double ratio = 1.0;
            for (int i = 1; i <= m; ++i) ratio *= (double)(M - i + 1) / (double)(M + i);
            const double a = 2.0 * ((m % 2) ? 1.0 : -1.0) * ratio / ((double)m * m);
            w[k] = a;
            centre -= 2.0 * dim * a;
        }
        w[0] = centre;
        return FD_OK;
    }
    if (d->scheme == FD_SPECTE_THETA || d->scheme == FD_DISPTE_THETA) {
        if (dim != 2) return set_error(FD_ERR_UNSUPPORTED, "theta schemes are defined for 2D only");
        std::vector<Orbit> sub;
        std::vector<int> idx;
        for (size_t k = 0; k < orbs.size(); ++k)
            if (d->scheme == FD_DISPTE_THETA || is_axis(orbs[k].key)) { sub.push_back(orbs[k]); idx.push_back((int)k); }
        Mat A;
        std::vector<dd> b;
        theta_system(sub, M, d->scheme == FD_DISPTE_THETA ? d->courant : 0.0, d->theta, A, b);
        std::vector<double> x;
        if (!dd_lstsq(A, b, x)) return set_error(FD_ERR_SINGULAR, "theta system is singular");
        for (size_t i = 0; i < idx.size(); ++i) w[idx[i]] = x[i];
        return FD_OK;
    }
    if (d->scheme == FD_DISPTE) {
        Mat A;
        std::vector<dd> b;
        moment_system(dim, orbs, M, d->courant, mixed_order(shape, M, N), A, b);
        std::vector<double> x;
        if (!dd_lstsq(A, b, x)) return set_error(FD_ERR_SINGULAR, "DispTE system is singular");
        w = x;
        return FD_OK;
    }
    st = ls_weights(dim, orbs, M, d->scheme, d->ls_basis, d->courant, d->band, w);
    if (st) return set_error(st, "least-squares design matrix is zero");
    return FD_OK;
}

double symbol_at(const std::vector<std::array<int, 3>> &offs, const std::vector<double> &wo,
                 const double k[3])
{
    double s = 0.0;
    for (size_t i = 0; i < offs.size(); ++i)
        s += wo[i] * std::cos(k[0] * offs[i][0] + k[1] * offs[i][1] + k[2] * offs[i][2]);
    return s;
}

// max over k in [0, pi]^dim of sign * S(k): a regular grid (corners included),
// then a compass pattern search from the best grid point.
static double symbol_extreme(const std::vector<std::array<int, 3>> &offs,
                             const std::vector<double> &wo, int dim, double sign, double kb[3])
{
    const int G = dim == 2 ? 97 : 33;
    double best = -1e300;
    kb[0] = kb[1] = kb[2] = 0.0;
    for (int a = 0; a < G; ++a)
        for (int bb = 0; bb < (dim == 3 ? G : 1); ++bb)
            for (int c = 0; c < G; ++c) {
                double k[3] = {kPi * a / (G - 1), dim == 3 ? kPi * bb / (G - 1) : 0.0, kPi * c / (G - 1)};
                const double v = sign * symbol_at(offs, wo, k);
                if (v > best) { best = v; std::memcpy(kb, k, 3 * sizeof(double)); }
            }
    double h = kPi / (G - 1);
    while (h > 1e-12) {
        bool moved = false;
        for (int ax = 0; ax < 3; ++ax) {
            if (dim == 2 && ax == 1) continue;
            for (int sgn = -1; sgn <= 1; sgn += 2) {
                double k[3] = {kb[0], kb[1], kb[2]};
                k[ax] = std::min(kPi, std::max(0.0, k[ax] + sgn * h));
                const double v = sign * symbol_at(offs, wo, k);
                if (v > best) { best = v; std::memcpy(kb, k, 3 * sizeof(double)); moved = true; }
            }
        }
        if (!moved) h *= 0.5;
    }
    return best;
}

// Von Neumann bound of the leapfrog (Eq. full_disp as the amplification
// equation lambda^2 - (2 + C^2 S) lambda + 1 = 0, whose roots have product 1):
// both roots lie on the unit circle iff -4 <= C^2 S(k) <= 0 for every k.  A
// symbol that is positive anywhere (beyond round-off: kSymbolPositiveTol of
// max -S; S(0) = 0 for a consistent stencil) is unstable at every time step.
int compute_cfl(const fd_stencil_desc *d, const std::vector<double> &w, double *cmax)
{
    std::vector<std::array<int, 3>> keys, offs;
    std::vector<int> mult, oo;
    std::vector<double> tmp;
    int st = compute_weights(d, keys, mult, tmp, &offs, &oo);
    if (st) return st;
    std::vector<double> wo(offs.size());
    for (size_t i = 0; i < offs.size(); ++i) wo[i] = w[oo[i]];
    const int dim = d->dim;
    constexpr double kSymbolPositiveTol = 1e-9;
    double kneg[3], kpos[3];
    const double neg = symbol_extreme(offs, wo, dim, -1.0, kneg);   // max -S
    const double pos = symbol_extreme(offs, wo, dim, +1.0, kpos);   // max S
    if (!(neg > 0.0)) return set_error(FD_ERR_UNSTABLE, "stencil symbol is non-negative: no stable time step");
    if (pos > kSymbolPositiveTol * neg)
        return set_error(FD_ERR_UNSTABLE,
                         "stencil symbol S(k) = %.6g > 0 at k h = (%.4f, %.4f, %.4f): the leapfrog is "
                         "unstable at every time step", pos, kpos[0], kpos[1], kpos[2]);
    *cmax = 2.0 / std::sqrt(neg);
    return FD_OK;
}

}  // namespace fdw

using namespace fdw;

extern "C" int fd_weights(const fd_stencil_desc *desc, int cap, int *n_orbits, int32_t *orbits,
                          int32_t *mult, double *w)
{
    clear_error();
    std::vector<std::array<int, 3>> keys;
    std::vector<int> m;
    std::vector<double> ww;
    int st = compute_weights(desc, keys, m, ww, nullptr, nullptr);
    if (st) return st;
    if (!n_orbits) return set_error(FD_ERR_ARG, "n_orbits is NULL");
    *n_orbits = (int)keys.size();
    if (cap < (int)keys.size()) return set_error(FD_ERR_ARG, "cap %d < %d orbits", cap, (int)keys.size());
    for (size_t i = 0; i < keys.size(); ++i) {
        if (orbits) for (int j = 0; j < 3; ++j) orbits[3 * i + j] = keys[i][j];
        if (mult) mult[i] = m[i];
        if (w) w[i] = ww[i];
    }
    return FD_OK;
}

extern "C" int fd_cfl_limit(const fd_stencil_desc *desc, double *courant_max)
{
    clear_error();
    if (!courant_max) return set_error(FD_ERR_ARG, "courant_max is NULL");
    std::vector<std::array<int, 3>> keys;
    std::vector<int> m;
    std::vector<double> w;
    int st = compute_weights(desc, keys, m, w, nullptr, nullptr);
    if (st) return st;
    return compute_cfl(desc, w, courant_max);
}

namespace {

// The min(m, n) largest singular values of a moment or theta system (dd
// entries rounded to double): an under-determined system (m < n) has no more
// than m non-zero ones.
std::vector<double> system_singular_values(const Mat &M)
{
    const int m = (int)M.size(), n = m ? (int)M[0].size() : 0;
    std::vector<double> a((size_t)m * n), V;
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j) a[(size_t)j * m + i] = M[i][j].hi + M[i][j].lo;
    jacobi_orthogonalise(a, m, n, V);
    std::vector<double> sig = column_norms(a, m, n);
    std::sort(sig.begin(), sig.end(), std::greater<double>());
    sig.resize(std::min(m, n));
    return sig;
}

}  // namespace

extern "C" int fd_weights_conditioning(const fd_stencil_desc *d, double *cond, int *rank,
                                       int *n_unknowns)
{
    clear_error();
    if (!cond || !rank || !n_unknowns) return set_error(FD_ERR_ARG, "NULL output");
    int st = check_desc(d);
    if (st) return st;
    const int dim = d->dim, M = d->M;
    auto orbs = build_orbits(dim, d->shape, M, d->N);
    auto is_axis = [](const std::array<int, 3> &k) { return k[1] == 0; };
    std::vector<double> sig;
    int r = 0, n_unk = 0;
    if (d->scheme == FD_SPECLS || d->scheme == FD_DISPLS) {
        std::vector<double> A, rhs;
        std::vector<int> cols;
        int m = 0, n = 0;
        ls_design(dim, orbs, M, d->scheme, d->ls_basis, d->courant, d->band, A, m, n, rhs, cols);
        std::vector<double> V;
        jacobi_orthogonalise(A, m, n, V);
        sig = column_norms(A, m, n);
        n_unk = n;
        const double smax = sig.empty() ? 0.0 : *std::max_element(sig.begin(), sig.end());
        for (double v : sig) r += v > kLsRcond * smax;
    } else {
        std::vector<Orbit> sub;
        for (auto &o : orbs)
            if (d->scheme == FD_DISPTE || d->scheme == FD_DISPTE_THETA || is_axis(o.key)) sub.push_back(o);
        Mat A;
        std::vector<dd> b;
        if (d->scheme == FD_SPECTE_THETA || d->scheme == FD_DISPTE_THETA) {
            if (dim != 2) return set_error(FD_ERR_UNSUPPORTED, "theta schemes are defined for 2D only");
            theta_system(sub, M, d->scheme == FD_DISPTE_THETA ? d->courant : 0.0, d->theta, A, b);
        } else if (d->scheme == FD_DISPTE) {
            moment_system(dim, sub, M, d->courant, mixed_order(d->shape, M, d->N), A, b);
        } else {   // SpatTE: the Taylor system of the axis orbits
            moment_system(dim, sub, M, 0.0, 1, A, b);
        }
        sig = system_singular_values(A);
        r = (int)independent_rows(A).size();
        n_unk = A.empty() ? 0 : (int)A[0].size();
    }
    const double smax = sig.empty() ? 0.0 : *std::max_element(sig.begin(), sig.end());
    const double smin = sig.empty() ? 0.0 : *std::min_element(sig.begin(), sig.end());
    *cond = smin > 0.0 ? smax / smin : HUGE_VAL;
    *rank = r;
    *n_unknowns = n_unk;
    return FD_OK;
}

extern "C" int fd_ricker(double f0, double dt, int nt, float *out)
{
    clear_error();
    if (!(f0 > 0) || !(dt > 0) || nt < 0 || (nt > 0 && !out))
        return set_error(FD_ERR_ARG, "fd_ricker needs f0 > 0, dt > 0, nt >= 0 and an output");
    for (int n = 0; n < nt; ++n) {
        const double a = kPi * f0 * (n * dt - 1.0 / f0);
        out[n] = (float)((1.0 - 2.0 * a * a) * std::exp(-a * a));
    }
    return FD_OK;
}
