// Step a0 of the hot path: from an equation of the form of Eq. (NPDE) to the
// polynomial coefficients of the equilibrium distribution f^eq_j(phi) that the
// kernels evaluate.  Host-only, double precision, no GPU.
//
// The auxiliary moments of Sec. II follow one pattern (Eqs. (Pi4), (Pi5), (Pi6)):
//     Pi_k0 = int_0^phi [ (Pi_1')^k + sum_{j=2}^{k-1} C(k,j) beta_j Pi_j' (Pi_1')^{k-j} + A_k0 ] dphi,
// with A_20 = A_30 = 0.  The inverse moment matrix M^-1 of Sec. III A/B is computed here
// exactly, in rationals, from the velocity set, and f^eq = M^-1 Pibar is folded into one
// polynomial per velocity.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "lbhpde.h"

namespace {

using Poly = std::vector<double>;  // Poly[p] = coefficient of phi^p

void trim(Poly &a) {
    while (!a.empty() && a.back() == 0.0) a.pop_back();
}
Poly mul(const Poly &a, const Poly &b) {
    if (a.empty() || b.empty()) return {};
    Poly r(a.size() + b.size() - 1, 0.0);
    for (size_t i = 0; i < a.size(); ++i)
        for (size_t j = 0; j < b.size(); ++j) r[i + j] += a[i] * b[j];
    return r;
}
void axpy(Poly &y, double s, const Poly &x) {
    if (s == 0.0) return;
    if (y.size() < x.size()) y.resize(x.size(), 0.0);
    for (size_t i = 0; i < x.size(); ++i) y[i] += s * x[i];
}
Poly deriv(const Poly &a) {
    if (a.size() <= 1) return {};
    Poly r(a.size() - 1);
    for (size_t i = 1; i < a.size(); ++i) r[i - 1] = double(i) * a[i];
    return r;
}
Poly integ0(const Poly &a) {  // int_0^phi, zero integration constant
    Poly r(a.size() + 1, 0.0);
    for (size_t i = 0; i < a.size(); ++i) r[i + 1] = a[i] / double(i + 1);
    return r;
}
bool is_zero(const Poly &a) {
    for (double v : a)
        if (v != 0.0) return false;
    return true;
}
bool is_phi(const Poly &a) {
    Poly t = a;
    trim(t);
    return t.size() == 2 && t[0] == 0.0 && t[1] == 1.0;
}

// Generalised polynomial in phi with one real exponent nu: sum_a (phi^nu)^a r[a](phi).  With one
// row it is an ordinary polynomial, and every operation below reduces to the Poly one exactly.
struct GPoly {
    std::vector<Poly> r;
};
void gtrim(GPoly &x) {
    for (auto &p : x.r) trim(p);
    while (!x.r.empty() && x.r.back().empty()) x.r.pop_back();
}
GPoly gmul(const GPoly &x, const GPoly &y) {
    GPoly t;
    if (x.r.empty() || y.r.empty()) return t;
    t.r.resize(x.r.size() + y.r.size() - 1);
    for (size_t a = 0; a < x.r.size(); ++a)
        for (size_t c = 0; c < y.r.size(); ++c) axpy(t.r[a + c], 1.0, mul(x.r[a], y.r[c]));
    return t;
}
void gaxpy(GPoly &y, double s, const GPoly &x) {
    if (s == 0.0) return;
    if (y.r.size() < x.r.size()) y.r.resize(x.r.size());
    for (size_t a = 0; a < x.r.size(); ++a) axpy(y.r[a], s, x.r[a]);
}
// d/dphi phi^(i + a nu) = (i + a nu) phi^(i - 1 + a nu); false if a term phi^(a nu), a >= 1, has
// no derivative of that form
bool gderiv(const GPoly &x, double nu, GPoly &out) {
    out.r.assign(x.r.size(), Poly{});
    for (size_t a = 0; a < x.r.size(); ++a) {
        const Poly &p = x.r[a];
        if (a >= 1 && !p.empty() && p[0] != 0.0) return false;
        if (p.size() <= 1) continue;
        Poly d(p.size() - 1);
        for (size_t i = 1; i < p.size(); ++i) d[i - 1] = (double(i) + double(a) * nu) * p[i];
        out.r[a] = d;
    }
    return true;
}
// int_0^phi: phi^(i + a nu) -> phi^(i + 1 + a nu) / (i + 1 + a nu)
GPoly ginteg0(const GPoly &x, double nu) {
    GPoly t;
    t.r.resize(x.r.size());
    for (size_t a = 0; a < x.r.size(); ++a) {
        Poly q(x.r[a].size() + 1, 0.0);
        for (size_t i = 0; i < x.r[a].size(); ++i) q[i + 1] = x.r[a][i] / (double(i + 1) + double(a) * nu);
        t.r[a] = q;
    }
    return t;
}
bool gis_zero(const GPoly &x) {
    for (const auto &p : x.r)
        if (!is_zero(p)) return false;
    return true;
}
bool gis_phi(const GPoly &x) {
    for (size_t a = 1; a < x.r.size(); ++a)
        if (!is_zero(x.r[a])) return false;
    return !x.r.empty() && is_phi(x.r[0]);
}

// Exact rational arithmetic for M^-1 (entries are small: denominators divide 720).
struct Q {
    int64_t n, d;
};
int64_t gcd64(int64_t a, int64_t b) {
    a = a < 0 ? -a : a;
    b = b < 0 ? -b : b;
    while (b) {
        int64_t t = a % b;
        a = b;
        b = t;
    }
    return a ? a : 1;
}
Q norm(Q a) {
    if (a.d < 0) a = {-a.n, -a.d};
    int64_t g = gcd64(a.n, a.d);
    return {a.n / g, a.d / g};
}
Q qsub(Q a, Q b) { return norm({a.n * b.d - b.n * a.d, a.d * b.d}); }
Q qmul(Q a, Q b) { return norm({a.n * b.n, a.d * b.d}); }
Q qdiv(Q a, Q b) { return norm({a.n * b.d, a.d * b.n}); }

// Inverse of the moment matrix M[k][j] = e_j^k (rows k = moment order, columns j = velocity),
// by Gauss-Jordan elimination in rationals.
void moment_matrix_inverse(int b, const int *e, double Minv[7][7]) {
    Q A[7][14];
    for (int k = 0; k < b; ++k) {
        for (int j = 0; j < b; ++j) {
            int64_t v = 1;
            for (int p = 0; p < k; ++p) v *= e[j];
            A[k][j] = {v, 1};
            A[k][b + j] = {k == j ? 1 : 0, 1};
        }
    }
    for (int col = 0; col < b; ++col) {
        int piv = col;
        while (A[piv][col].n == 0) ++piv;  // M is a non-singular Vandermonde matrix
        if (piv != col)
            for (int j = 0; j < 2 * b; ++j) std::swap(A[piv][j], A[col][j]);
        Q p = A[col][col];
        for (int j = 0; j < 2 * b; ++j) A[col][j] = qdiv(A[col][j], p);
        for (int r = 0; r < b; ++r) {
            if (r == col || A[r][col].n == 0) continue;
            Q f = A[r][col];
            for (int j = 0; j < 2 * b; ++j) A[r][j] = qsub(A[r][j], qmul(f, A[col][j]));
        }
    }
    for (int i = 0; i < b; ++i)
        for (int j = 0; j < b; ++j) Minv[i][j] = double(A[i][b + j].n) / double(A[i][b + j].d);
}

double binom(int n, int k) {
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * double(n - k + i) / double(i);
    return r;
}

bool near_zero(double x) { return std::fabs(x) < 1e-13; }

int pi_to_poly(const lbhpde_pi &p, Poly &out);

// Pi_k as a generalised polynomial; nu: the equation's real exponent so far (0 = none yet),
// set or checked by a LBHPDE_PI_POLY_NU term.
int pi_to_gpoly(const lbhpde_pi &p, double &nu, GPoly &out) {
    out.r.clear();
    Poly row0;
    if (p.kind != LBHPDE_PI_POLY_NU) {
        int rc = pi_to_poly(p, row0);
        if (rc) return rc;
        out.r.push_back(row0);
        return LBHPDE_OK;
    }
    if (!(p.nu > 0.0) || !std::isfinite(p.nu) || p.nu > 64.0) return LBHPDE_ERR_ARG;
    if (nu != 0.0 && nu != p.nu) return LBHPDE_ERR_ARG;  // one real exponent per equation
    nu = p.nu;
    if (p.coef_nu[0] != 0.0) return LBHPDE_ERR_ARG;  // phi^nu would have no derivative of the form
    row0.assign(p.coef, p.coef + LBHPDE_PI_NCOEF);
    Poly row1(p.coef_nu, p.coef_nu + LBHPDE_PI_NCOEF);
    for (double v : row0)
        if (!std::isfinite(v)) return LBHPDE_ERR_ARG;
    for (double v : row1)
        if (!std::isfinite(v)) return LBHPDE_ERR_ARG;
    out.r = {row0, row1};
    gtrim(out);
    return LBHPDE_OK;
}

int pi_to_poly(const lbhpde_pi &p, Poly &out) {
    out.clear();
    switch (p.kind) {
    case LBHPDE_PI_ZERO:
        return LBHPDE_OK;
    case LBHPDE_PI_PHI:
        out = {0.0, 1.0};
        return LBHPDE_OK;
    case LBHPDE_PI_POWER:
        if (p.power < 1 || p.power > 7) return LBHPDE_ERR_ARG;
        out.assign(p.power + 1, 0.0);
        out[p.power] = 1.0;
        return LBHPDE_OK;
    case LBHPDE_PI_POLY:
        out.assign(p.coef, p.coef + LBHPDE_PI_NCOEF);
        for (double v : out)
            if (!std::isfinite(v)) return LBHPDE_ERR_ARG;
        trim(out);
        return LBHPDE_OK;
    default:
        return LBHPDE_ERR_ARG;
    }
}

}  // namespace

// The velocity order shared by the whole library: e = {0, 1, -1, 2, -2, 3, -3}.
static const int kVel[7] = {0, 1, -1, 2, -2, 3, -3};

extern "C" int lbhpde_model(int m, const double *alpha, const lbhpde_pi *pi, double dx, double dt,
                            double tau, int lattice, int scheme, lbhpde_model_info *out) {
    if (!out || !alpha || !pi) return LBHPDE_ERR_ARG;
    std::memset(out, 0, sizeof(*out));
    if (m < 1 || m > 6) return LBHPDE_ERR_ARG;
    if (!(dx > 0.0) || !(dt > 0.0) || !(tau > 0.0) || !std::isfinite(dx) || !std::isfinite(dt) ||
        !std::isfinite(tau))
        return LBHPDE_ERR_ARG;
    const int b = lattice == 0 ? (m <= 4 ? 5 : 7) : lattice;
    if (b != 5 && b != 7) return LBHPDE_ERR_ARG;
    if (m > b - 1) return LBHPDE_ERR_ARG;  // at least m + 1 velocities (Sec. III)
    const bool no_aux = (scheme & LBHPDE_NO_AUX_CORRECTION) != 0;
    scheme &= ~LBHPDE_NO_AUX_CORRECTION;
    if (scheme != 1 && scheme != 2) return LBHPDE_ERR_ARG;
    if (scheme == 2 && m >= b - 1) return LBHPDE_ERR_ARG;
    for (int k = 0; k < m; ++k)
        if (!std::isfinite(alpha[k])) return LBHPDE_ERR_ARG;

    const double c = dx / dt;
    // Pi_1..Pi_6 (index 1..6); alpha_1 folded into Pi_1.
    GPoly P[7];
    double nu = 0.0;
    for (int k = 1; k <= m; ++k) {
        int rc = pi_to_gpoly(pi[k - 1], nu, P[k]);
        if (rc) return rc;
    }
    for (auto &row : P[1].r)
        for (double &v : row) v *= alpha[0];

    // Eq. (taus), evaluated by Horner's rule in tau.
    double tk[7] = {0.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    tk[2] = 0.5 - tau;
    tk[3] = 1.0 / 6.0 + tau * (-1.0 + tau);
    tk[4] = 1.0 / 24.0 + tau * (-7.0 / 12.0 + tau * (1.5 - tau));
    tk[5] = 1.0 / 120.0 + tau * (-0.25 + tau * (1.25 + tau * (-2.0 + tau)));
    tk[6] = 1.0 / 720.0 + tau * (-31.0 / 360.0 + tau * (0.75 + tau * (-13.0 / 6.0 + tau * (2.5 - tau))));

    // alpha_k = dt^{k-1} tau_k beta_k; a term that is absent takes beta_k = 0 (Remark 2).
    double beta[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int k = 2; k <= m; ++k) {
        if (alpha[k - 1] == 0.0 || gis_zero(P[k])) continue;
        if (near_zero(tk[k])) return LBHPDE_ERR_TAU_SINGULAR;
        beta[k] = alpha[k - 1] / (std::pow(dt, double(k - 1)) * tk[k]);
    }

    // A_k0 of Eqs. (Pi4)-(Pi6); only moments the lattice carries need them.  With
    // LBHPDE_NO_AUX_CORRECTION they are left out, and recovery is flagged inexact wherever
    // one of them would be present.
    double A[7] = {0, 0, 0, 0, 0, 0, 0};
    const bool need4 = b - 1 >= 4 && beta[2] != 0.0;
    const bool need5 = b - 1 >= 5 && beta[2] != 0.0 && beta[3] != 0.0;
    const bool need6 = b - 1 >= 6 && (beta[2] != 0.0 || beta[3] != 0.0);
    if (!no_aux) {
        if (need4) {
            if (near_zero(tk[4])) return LBHPDE_ERR_TAU_SINGULAR;
            A[4] = tk[2] * (3.0 * tk[3] - tk[2] * tk[2]) * beta[2] * beta[2] / tk[4];
        }
        if (need5) {
            if (near_zero(tk[5])) return LBHPDE_ERR_TAU_SINGULAR;
            A[5] = (4.0 * tk[2] * tk[4] + 3.0 * tk[3] * tk[3] - 2.0 * tk[2] * tk[2] * tk[3]) * beta[2] *
                   beta[3] / tk[5];
        }
        if (need6) {
            if (near_zero(tk[6])) return LBHPDE_ERR_TAU_SINGULAR;
            const double t2 = tk[2], t3 = tk[3], t4 = tk[4], t5 = tk[5];
            A[6] = ((5.0 * t2 * t5 + 3.0 * t3 * t4 - 2.0 * t2 * t2 * t4) * beta[2] * beta[4] +
                    (4.0 * t4 - t2 * t3) * t3 * beta[3] * beta[3] +
                    (t2 * t3 - 6.0 * t4) * t2 * t2 * beta[2] * beta[2] * beta[2]) /
                   tk[6];
        }
    }

    // Exact-recovery preconditions (Sec. II D-F, Remarks 2, 4, 5).
    int inexact = 0;
    if (b - 1 >= 4 && beta[2] != 0.0 && !gis_phi(P[2])) inexact = 1;
    if (b - 1 >= 5 && beta[2] != 0.0 && beta[3] != 0.0 && !(gis_phi(P[2]) && gis_phi(P[3]))) inexact = 1;
    if (b - 1 >= 6 && beta[3] != 0.0 && !gis_phi(P[3])) inexact = 1;
    if (b - 1 >= 6 && beta[2] != 0.0 && beta[4] != 0.0 && !(gis_phi(P[2]) && gis_phi(P[4]))) inexact = 1;
    if (b == 7 && beta[2] != 0.0) inexact = 1;
    if (no_aux && (need4 || need5 || need6)) inexact = 1;

    // Auxiliary moments Pi_k0, k = 2..b-1 (beta_k = 0 for k > m).
    GPoly d1;
    if (!gderiv(P[1], nu, d1)) return LBHPDE_ERR_ARG;
    GPoly d1pow[7];
    d1pow[0].r = {Poly{1.0}};
    for (int k = 1; k <= 6; ++k) d1pow[k] = gmul(d1pow[k - 1], d1);
    GPoly Pibar[7];
    Pibar[0].r = {Poly{0.0, 1.0}};
    Pibar[1] = P[1];
    for (auto &row : Pibar[1].r)
        for (double &v : row) v /= c;
    for (int k = 2; k < b; ++k) {
        GPoly g = d1pow[k];
        for (int j = 2; j <= k - 1; ++j) {
            if (beta[j] == 0.0) continue;
            GPoly dj;
            if (!gderiv(P[j], nu, dj)) return LBHPDE_ERR_ARG;
            gaxpy(g, binom(k, j) * beta[j], gmul(dj, d1pow[k - j]));
        }
        GPoly one;
        one.r = {Poly{1.0}};
        gaxpy(g, A[k], one);
        GPoly Pk0 = ginteg0(g, nu);
        gaxpy(Pk0, beta[k], P[k]);
        const double ck = std::pow(c, double(k));
        for (auto &row : Pk0.r)
            for (double &v : row) v /= ck;
        Pibar[k] = Pk0;
    }
    if (scheme == 2) Pibar[b - 1].r.clear();

    double Minv[7][7];
    moment_matrix_inverse(b, kVel, Minv);
    int Dg = 0, rows = 1;
    GPoly feq[7];
    for (int j = 0; j < b; ++j) {
        for (int k = 0; k < b; ++k) gaxpy(feq[j], Minv[j][k], Pibar[k]);
        gtrim(feq[j]);
        rows = std::max(rows, (int)feq[j].r.size());
        for (const auto &row : feq[j].r) Dg = std::max(Dg, (int)row.size() - 1);
    }
    if (rows == 1) nu = 0.0;  // no real-exponent term survives: an ordinary polynomial model
    int D = Dg;
    if (rows == 1 && D > LBHPDE_MAX_DEG) return LBHPDE_ERR_ARG;
    if (rows > 1) {
        if (rows * (Dg + 1) > LBHPDE_NU_TERMS) return LBHPDE_ERR_ARG;
        D = rows * (Dg + 1) - 1;
    }

    out->b = b;
    out->m = m;
    out->scheme = scheme;
    out->D = D;
    out->inexact = inexact;
    out->c = c;
    out->omega = 1.0 / tau;
    for (int k = 0; k < 7; ++k) {
        out->tk[k] = k >= 2 ? tk[k] : 0.0;
        out->beta[k] = beta[k];
    }
    out->A[0] = A[4];
    out->A[1] = A[5];
    out->A[2] = A[6];
    out->nu = nu;
    out->nu_rows = rows;
    out->nu_deg = Dg;
    for (int j = 0; j < b; ++j)
        for (size_t a = 0; a < feq[j].r.size(); ++a)
            for (size_t p = 0; p < feq[j].r[a].size(); ++p) {
                const double v = feq[j].r[a][p];
                out->gfeq[j][a * (Dg + 1) + p] = v;
                out->gcoef[j][a * (Dg + 1) + p] = v / tau;
                if (rows == 1) {
                    out->feq[j][p] = v;
                    out->coef[j][p] = v / tau;
                }
            }
    return LBHPDE_OK;
}

extern "C" const char *lbhpde_strerror(int code) {
    switch (code) {
    case LBHPDE_OK: return "ok";
    case LBHPDE_ERR_ARG: return "invalid argument";
    case LBHPDE_ERR_TAU_SINGULAR: return "singular relaxation time: tau_k = 0 where beta_k or A_k0 needs it";
    case LBHPDE_ERR_OOM: return "device memory exhausted or over budget";
    case LBHPDE_ERR_DIVERGED: return "non-finite phi (the scheme diverged)";
    case LBHPDE_PENDING: return "pending";
    case LBHPDE_ERR_TIMEOUT: return "timed out";
    case LBHPDE_ERR_CUDA: return "CUDA runtime error";
    case LBHPDE_ERR_NOT_FOUND: return "unknown request";
    case LBHPDE_ERR_UNSUPPORTED: return "not supported by this kernel";
    default: return "unknown status";
    }
}
