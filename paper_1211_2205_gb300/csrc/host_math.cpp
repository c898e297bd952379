// Host mathematics of the StaRMAP stepper (FP64).
//
// Moment matrices (section 3 of Seibold & Frank, arXiv:1211.2205): the
// complex P_N matrices are read off eq. Pncomplex using the recursion
// coefficients a..f of section 3; the real matrices follow as S M S^-1 with
// the unitary S of eq. transformation.  S has at most two nonzeros per row,
// so M^real[r][c] = sum over a in supp S_r, b in supp S_c of
// S[r][a] M^c[a][b] conj(S[c][b]) is evaluated sparsely.
//
// Grid placement follows eq. matrix_conditions: component 0 (R_0^0) goes to
// G11 and every nonzero of Mx (My) places a partner on the grid staggered in
// x (y) (section 5.3).  lambda_max(Mx) (section 5.3) is found per connected
// block by Householder tridiagonalisation and Sturm-sequence bisection.
#include "host_math.h"

#include <cmath>
#include <complex>
#include <deque>
#include <map>
#include <utility>

namespace starmap {

namespace {

using cplx = std::complex<double>;

double radicand_sqrt(double num, double den) {
    double q = num / den;
    return q <= 0.0 ? 0.0 : std::sqrt(q);
}
// Recursion coefficients of section 3 (Brunner & Holloway form).
double rc_c(int l, int m) { return radicand_sqrt(double(l + m + 1) * (l + m + 2), double(2 * l + 3) * (2 * l + 1)); }
double rc_d(int l, int m) { return radicand_sqrt(double(l - m) * (l - m - 1), double(2 * l + 1) * (2 * l - 1)); }
double rc_e(int l, int m) { return radicand_sqrt(double(l - m + 1) * (l - m + 2), double(2 * l + 3) * (2 * l + 1)); }
double rc_f(int l, int m) { return radicand_sqrt(double(l + m) * (l + m - 1), double(2 * l + 1) * (2 * l - 1)); }

struct SparseC {   // sparse complex matrix as map (row, col) -> value
    std::map<std::pair<int, int>, cplx> v;
    void add(int r, int c, cplx x) { v[{r, c}] += x; }
};

void build_pn2d(int N, SystemMatrices& out) {
    // complex moments (l, m), l + m even (z-symmetry, section 3)
    std::map<std::pair<int, int>, int> cidx;
    int nc = 0;
    for (int l = 0; l <= N; ++l)
        for (int m = -l; m <= l; ++m)
            if (((l + m) % 2 + 2) % 2 == 0) cidx[{l, m}] = nc++;
    auto has = [&](int l, int m) { return cidx.count({l, m}) != 0; };

    // eq. Pncomplex: row (l, m) couples to (l-1, m-1), (l+1, m-1), (l-1, m+1), (l+1, m+1)
    SparseC Mxc, Myc;
    const cplx I(0.0, 1.0);
    for (auto& kv : cidx) {
        int l = kv.first.first, m = kv.first.second, row = kv.second;
        if (has(l - 1, m - 1)) {
            double c = rc_c(l - 1, m - 1);
            Mxc.add(row, cidx[{l - 1, m - 1}], -0.5 * c);
            Myc.add(row, cidx[{l - 1, m - 1}], 0.5 * I * c);
        }
        if (has(l + 1, m - 1)) {
            double d = rc_d(l + 1, m - 1);
            Mxc.add(row, cidx[{l + 1, m - 1}], 0.5 * d);
            Myc.add(row, cidx[{l + 1, m - 1}], -0.5 * I * d);
        }
        if (has(l - 1, m + 1)) {
            double e = rc_e(l - 1, m + 1);
            Mxc.add(row, cidx[{l - 1, m + 1}], 0.5 * e);
            Myc.add(row, cidx[{l - 1, m + 1}], 0.5 * I * e);
        }
        if (has(l + 1, m + 1)) {
            double f = rc_f(l + 1, m + 1);
            Mxc.add(row, cidx[{l + 1, m + 1}], -0.5 * f);
            Myc.add(row, cidx[{l + 1, m + 1}], -0.5 * I * f);
        }
    }

    // real moments in the order of eq. transformation and their S rows
    struct Srow { int n = 0; int col[2]; cplx val[2]; };
    std::vector<Srow> S;
    out.moms.clear();
    const double r2 = 1.0 / std::sqrt(2.0);
    for (int l = 0; l <= N; ++l) {
        for (int m = l; m > 0; m -= 2) {
            double sg = (m % 2) ? -1.0 : 1.0;
            Srow R, Im;
            R.n = 2; R.col[0] = cidx[{l, m}]; R.val[0] = sg * r2; R.col[1] = cidx[{l, -m}]; R.val[1] = r2;
            Im.n = 2; Im.col[0] = cidx[{l, m}]; Im.val[0] = I * sg * r2; Im.col[1] = cidx[{l, -m}]; Im.val[1] = -I * r2;
            Moment a; a.l = l; a.m = m; a.imag = false; out.moms.push_back(a); S.push_back(R);
            Moment b; b.l = l; b.m = m; b.imag = true;  out.moms.push_back(b); S.push_back(Im);
        }
        if (l % 2 == 0) {
            Srow R; R.n = 1; R.col[0] = cidx[{l, 0}]; R.val[0] = 1.0;
            Moment a; a.l = l; a.m = 0; a.imag = false; out.moms.push_back(a); S.push_back(R);
        }
    }
    int n = (int)out.moms.size();
    out.ncomp = n;
    // column lookup: complex index -> list of (real row, S value)
    std::vector<std::vector<std::pair<int, cplx>>> colmap(nc);
    for (int r = 0; r < n; ++r)
        for (int t = 0; t < S[r].n; ++t) colmap[S[r].col[t]].push_back({r, S[r].val[t]});

    for (int which = 0; which < 2; ++which) {
        const SparseC& Mc = which == 0 ? Mxc : Myc;
        std::vector<cplx> acc((size_t)n * n, cplx(0.0));
        // M^real = S Mc S^H : for every Mc(a,b): rows r with S[r][a], cols c with S[c][b]
        for (auto& kv : Mc.v) {
            int a = kv.first.first, b = kv.first.second;
            for (auto& ra : colmap[a])
                for (auto& cb : colmap[b])
                    acc[(size_t)ra.first * n + cb.first] += ra.second * kv.second * std::conj(cb.second);
        }
        std::vector<double>& M = which == 0 ? out.Mx : out.My;
        M.assign((size_t)n * n, 0.0);
        for (size_t k = 0; k < acc.size(); ++k) {
            double re = acc[k].real();
            M[k] = std::fabs(re) < 1e-13 ? 0.0 : re;
        }
    }
}

void build_slab(int N, SystemMatrices& out) {
    int n = N + 1;
    out.ncomp = n;
    out.moms.clear();
    for (int l = 0; l <= N; ++l) { Moment a; a.l = l; a.m = 0; out.moms.push_back(a); }
    out.Mx.assign((size_t)n * n, 0.0);
    out.My.assign((size_t)n * n, 0.0);
    for (int l = 0; l <= N; ++l) {          // eq. PN_slab
        if (l + 1 <= N) out.Mx[(size_t)l * n + l + 1] = double(l + 1) / (2 * l + 1);
        if (l - 1 >= 0) out.Mx[(size_t)l * n + l - 1] = double(l) / (2 * l + 1);
    }
}

bool place_on_grids(SystemMatrices& s, std::string& err) {
    int n = s.ncomp;
    std::vector<int> gx(n, 0), gy(n, 0);
    gx[0] = 1; gy[0] = 1;
    std::deque<int> q{0};
    while (!q.empty()) {
        int i = q.front(); q.pop_front();
        for (int j = 0; j < n; ++j) {
            for (int which = 0; which < 2; ++which) {
                const std::vector<double>& M = which == 0 ? s.Mx : s.My;
                if (M[(size_t)i * n + j] == 0.0 && M[(size_t)j * n + i] == 0.0) continue;
                int wx = which == 0 ? 3 - gx[i] : gx[i];
                int wy = which == 0 ? gy[i] : 3 - gy[i];
                if (gx[j] == 0) { gx[j] = wx; gy[j] = wy; q.push_back(j); }
                else if (gx[j] != wx || gy[j] != wy) { err = "coupling pattern admits no staggered placement"; return false; }
            }
        }
    }
    for (int g = 0; g < 4; ++g) s.grid_count[g] = 0;
    for (int j = 0; j < n; ++j) {
        if (gx[j] == 0) { err = "component not reachable from R_0^0"; return false; }
        int g = (gx[j] - 1) + 2 * (gy[j] - 1);       // 0 G11, 1 G21, 2 G12, 3 G22
        s.moms[j].grid = g;
        s.moms[j].local = s.grid_count[g]++;
    }
    return true;
}

// Householder reduction of a dense symmetric matrix to tridiagonal form.
void tridiagonalise(std::vector<double> A, int n, std::vector<double>& d, std::vector<double>& e) {
    d.assign(n, 0.0);
    e.assign(n, 0.0);
    for (int k = 0; k < n - 2; ++k) {
        double alpha = 0.0;
        for (int i = k + 1; i < n; ++i) alpha += A[(size_t)i * n + k] * A[(size_t)i * n + k];
        alpha = std::sqrt(alpha);
        if (alpha == 0.0) continue;
        double x0 = A[(size_t)(k + 1) * n + k];
        if (x0 > 0) alpha = -alpha;
        std::vector<double> v(n, 0.0);
        v[k + 1] = x0 - alpha;
        for (int i = k + 2; i < n; ++i) v[i] = A[(size_t)i * n + k];
        double vn = 0.0;
        for (int i = k + 1; i < n; ++i) vn += v[i] * v[i];
        if (vn == 0.0) continue;
        // A <- H A H with H = I - 2 v v^T / vn ;  p = A v, K = v^T p / vn, w = 2(p - K v)/vn
        std::vector<double> p(n, 0.0);
        for (int i = k; i < n; ++i) {
            double s = 0.0;
            for (int j = k + 1; j < n; ++j) s += A[(size_t)i * n + j] * v[j];
            p[i] = s;
        }
        double K = 0.0;
        for (int i = k + 1; i < n; ++i) K += v[i] * p[i];
        K /= vn;
        std::vector<double> w(n, 0.0);
        for (int i = k; i < n; ++i) w[i] = 2.0 * (p[i] - K * v[i]) / vn;
        for (int i = k; i < n; ++i)
            for (int j = k; j < n; ++j)
                A[(size_t)i * n + j] -= v[i] * w[j] + w[i] * v[j];
    }
    for (int i = 0; i < n; ++i) d[i] = A[(size_t)i * n + i];
    for (int i = 0; i + 1 < n; ++i) e[i] = A[(size_t)(i + 1) * n + i];
}

// number of eigenvalues of the tridiagonal (d, e) strictly below x
int sturm_count(const std::vector<double>& d, const std::vector<double>& e, double x) {
    int n = (int)d.size(), cnt = 0;
    double q = 1.0;
    for (int i = 0; i < n; ++i) {
        double off = i > 0 ? e[i - 1] * e[i - 1] : 0.0;
        q = d[i] - x - (i > 0 ? off / q : 0.0);
        if (q == 0.0) q = -1e-300;
        if (q < 0.0) ++cnt;
    }
    return cnt;
}

double tridiagonal_extreme(const std::vector<double>& d, const std::vector<double>& e, bool largest) {
    int n = (int)d.size();
    double bound = 0.0;
    for (int i = 0; i < n; ++i) {
        double r = std::fabs(d[i]) + (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i + 1 < n ? std::fabs(e[i]) : 0.0);
        bound = std::max(bound, r);
    }
    double lo = -bound - 1e-300, hi = bound + 1e-300;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid == lo || mid == hi) break;
        int c = sturm_count(d, e, mid);
        if (largest) { if (c < n) lo = mid; else hi = mid; }      // some eigenvalue >= mid
        else         { if (c >= 1) hi = mid; else lo = mid; }     // some eigenvalue < mid
    }
    return 0.5 * (lo + hi);
}

}  // namespace

double symmetric_spectral_radius(const std::vector<double>& A, int n) {
    // split into connected blocks of the nonzero graph; each block separately
    std::vector<int> comp(n, -1);
    int ncomp = 0;
    for (int s = 0; s < n; ++s) {
        if (comp[s] >= 0) continue;
        std::deque<int> q{s};
        comp[s] = ncomp;
        while (!q.empty()) {
            int i = q.front(); q.pop_front();
            for (int j = 0; j < n; ++j)
                if (comp[j] < 0 && (A[(size_t)i * n + j] != 0.0 || A[(size_t)j * n + i] != 0.0)) {
                    comp[j] = ncomp; q.push_back(j);
                }
        }
        ++ncomp;
    }
    double rho = 0.0;
    for (int c = 0; c < ncomp; ++c) {
        std::vector<int> idx;
        for (int i = 0; i < n; ++i) if (comp[i] == c) idx.push_back(i);
        int m = (int)idx.size();
        if (m == 1) { rho = std::max(rho, std::fabs(A[(size_t)idx[0] * n + idx[0]])); continue; }
        std::vector<double> B((size_t)m * m);
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) B[(size_t)i * m + j] = A[(size_t)idx[i] * n + idx[j]];
        std::vector<double> d, e;
        tridiagonalise(B, m, d, e);
        rho = std::max(rho, std::fabs(tridiagonal_extreme(d, e, true)));
        rho = std::max(rho, std::fabs(tridiagonal_extreme(d, e, false)));
    }
    return rho;
}

double expm1div(double c) {
    // section 5.6: series 1 + c/2 + c^2/6 near zero (the printed line is E(-c))
    if (std::fabs(c) <= 2e-4) return 1.0 + c / 2.0 + c * c / 6.0;
    return std::expm1(c) / c;
}

bool build_system(int system, int N, SystemMatrices& out, std::string& err) {
    if (N < 0 || N > 63) { err = "moment order N must be in [0, 63]"; return false; }
    out.system = system;
    out.N = N;
    if (system == 0) build_pn2d(N, out);
    else if (system == 1) build_slab(N, out);
    else { err = "unknown system"; return false; }
    if (!place_on_grids(out, err)) return false;
    int n = out.ncomp;
    if (system == 0) {
        out.lambda_max = symmetric_spectral_radius(out.Mx, n);
    } else {
        // tridiagonal with positive products: similar to the symmetric matrix
        // with off-diagonals sqrt(M[l][l+1] M[l+1][l])
        std::vector<double> Sym((size_t)n * n, 0.0);
        for (int l = 0; l + 1 < n; ++l) {
            double v = std::sqrt(out.Mx[(size_t)l * n + l + 1] * out.Mx[(size_t)(l + 1) * n + l]);
            Sym[(size_t)l * n + l + 1] = v;
            Sym[(size_t)(l + 1) * n + l] = v;
        }
        out.lambda_max = symmetric_spectral_radius(Sym, n);
    }
    if (n == 1) out.lambda_max = 0.0;
    return true;
}

// The real harmonic of every component at the direction (mu, phi): the
// orthonormal associated Legendre functions N_l^m P_l^m(mu) without the
// Condon-Shortley phase (so R_1^1 ~ Omega_x, I_1^1 ~ Omega_y, the convention
// of the real moments of section 3), by the standard three-term recurrence
// in l at fixed m, started from N_m^m P_m^m = sqrt(1/(4 pi)) prod_k
// sqrt((2k+1)/(2k)) (1 - mu^2)^(m/2); then R_l^m = sqrt2 Ybar cos(m phi),
// I_l^m = sqrt2 Ybar sin(m phi), R_l^0 = Ybar.
bool direction_moments(int system, int N, double mu, double phi, std::vector<double>& out, std::string& err) {
    if (system != 0) { err = "direction moments are defined for the 2D system"; return false; }
    if (!(mu >= -1.0 && mu <= 1.0)) { err = "mu must lie in [-1, 1]"; return false; }
    SystemMatrices sys;
    if (!build_system(system, N, sys, err)) return false;
    const double pi = std::acos(-1.0);
    const double st = std::sqrt(std::max(0.0, 1.0 - mu * mu));
    // ybar[m][l]: orthonormal associated Legendre values
    std::vector<std::vector<double>> ybar(N + 1, std::vector<double>(N + 1, 0.0));
    double ymm = std::sqrt(1.0 / (4.0 * pi));
    for (int m = 0; m <= N; ++m) {
        if (m > 0) ymm *= std::sqrt((2.0 * m + 1.0) / (2.0 * m)) * st;
        ybar[m][m] = ymm;
        if (m + 1 <= N) ybar[m][m + 1] = std::sqrt(2.0 * m + 3.0) * mu * ymm;
        for (int l = m + 2; l <= N; ++l) {
            const double a = std::sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
            const double b = std::sqrt(((l - 1.0) * (l - 1.0) - (double)m * m) / (4.0 * (l - 1.0) * (l - 1.0) - 1.0));
            ybar[m][l] = a * (mu * ybar[m][l - 1] - b * ybar[m][l - 2]);
        }
    }
    out.assign(sys.ncomp, 0.0);
    for (int j = 0; j < sys.ncomp; ++j) {
        const Moment& mo = sys.moms[j];
        const double y = ybar[mo.m][mo.l];
        if (mo.m == 0) out[j] = y;
        else out[j] = std::sqrt(2.0) * y * (mo.imag ? std::sin(mo.m * phi) : std::cos(mo.m * phi));
    }
    return true;
}

}  // namespace starmap
