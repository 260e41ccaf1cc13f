// Offline stage of Polar Express: greedy minimax coefficient table in FP64.
//
// Thm. 1 (Eq. greedy, Eq. newbounds): p_t is the minimax odd polynomial for
// x -> 1 on [l_t, u_t]; l_{t+1} = p_t(l_t), u_{t+1} = 2 - l_{t+1}.
// Degree 5 uses the simplified Remez iteration of Alg. 3 (App. F): trial set
// {l, x1, x2, u}; solve the 4x4 alternation system for (a, b, c, E); move
// x1, x2 to the roots of p'(x) = a + 3b x^2 + 5c x^4; stop when E stops
// changing. Degree 3 uses the closed form Eq. deg3_solution. Stabilisation
// (Sec. 3.4, App. G, App. A offline code): cushioned interval
// [max(l_t, kappa u_t), u_t], recentring by 2 / (p(l_t) + max p), and the
// safety factor p_t(x / s) on every row not taken from the l/u -> 1 shortcut.
//
// Compiled with -ffp-contract=off and without fast-math: every product and
// sum below is one IEEE double operation in the written order, so the table
// is reproducible bit for bit on any conforming host.
#include <cmath>
#include <cstring>
#include <limits>

#include "pe_internal.h"

namespace pe {
namespace {

constexpr double kKappa5 = 0.02407327424182761;
constexpr double kKappa3 = 0.1;
constexpr double kShortcut = 1.0 - 5e-6;
constexpr double kRemezTol = 1e-15;
constexpr int kRemezMaxIters = 100;

inline double cube(double x) { return x * x * x; }
inline double fifth(double x) { return x * x * x * x * x; }
inline double odd5(double a, double b, double c, double x) {
    return a * x + b * cube(x) + c * fifth(x);
}

// Gaussian elimination with partial pivoting on an augmented 4x5 system:
// the first row holding the largest |pivot| is swapped up, rows below are
// eliminated in natural order, then back substitution from the last row.
bool solve4(double A[4][5], double z[4]) {
    for (int k = 0; k < 4; ++k) {
        int p = k;
        double best = std::fabs(A[k][k]);
        for (int i = k + 1; i < 4; ++i) {
            double v = std::fabs(A[i][k]);
            if (v > best) { best = v; p = i; }
        }
        if (best == 0.0) return false;
        if (p != k) {
            for (int j = 0; j < 5; ++j) { double t = A[k][j]; A[k][j] = A[p][j]; A[p][j] = t; }
        }
        const double piv = A[k][k];
        for (int i = k + 1; i < 4; ++i) {
            const double f = A[i][k] / piv;
            for (int j = k + 1; j < 5; ++j) A[i][j] = A[i][j] - f * A[k][j];
        }
    }
    for (int i = 3; i >= 0; --i) {
        double acc = A[i][4];
        for (int j = i + 1; j < 4; ++j) acc = acc - A[i][j] * z[j];
        z[i] = acc / A[i][i];
    }
    return true;
}

struct Quintic { double a, b, c; bool shortcut; int iters; };

// Minimax odd quintic on [lo, hi]; returns PE_OK / PE_ENOCONV / PE_EINVAL.
int minimax_quintic(double lo, double hi, Quintic* q) {
    if (!(lo > 0.0 && hi > 0.0)) return PE_EINVAL;
    if (lo / hi >= kShortcut) {
        // (x/u)(15 - 10 (x/u)^2 + 3 (x/u)^4) / 8, the Newton-Schulz limit.
        q->a = (15.0 / 8.0) / hi;
        q->b = (-10.0 / 8.0) / cube(hi);
        q->c = (3.0 / 8.0) / fifth(hi);
        q->shortcut = true;
        q->iters = 0;
        return PE_OK;
    }
    double x1 = (3.0 * lo + hi) / 4.0;
    double x2 = (lo + 3.0 * hi) / 4.0;
    double E = std::numeric_limits<double>::infinity();
    bool first = true;
    double E_prev = 0.0;
    double a = 0, b = 0, c = 0;
    int it = 0;
    while (first || std::fabs(E_prev - E) > kRemezTol) {
        if (it >= kRemezMaxIters) return PE_ENOCONV;
        first = false;
        E_prev = E;
        const double pts[4] = {lo, x1, x2, hi};
        double M[4][5];
        for (int r = 0; r < 4; ++r) {
            const double x = pts[r];
            M[r][0] = x;
            M[r][1] = cube(x);
            M[r][2] = fifth(x);
            M[r][3] = (r % 2 == 0) ? 1.0 : -1.0;
            M[r][4] = 1.0;
        }
        double z[4];
        if (!solve4(M, z)) return PE_ENOCONV;
        a = z[0]; b = z[1]; c = z[2]; E = z[3];
        const double disc = 9.0 * (b * b) - 20.0 * a * c;
        const double sq = std::sqrt(disc);
        x1 = std::sqrt((-3.0 * b - sq) / (10.0 * c));
        x2 = std::sqrt((-3.0 * b + sq) / (10.0 * c));
        ++it;
        if (!std::isfinite(x1) || !std::isfinite(x2)) return PE_ENOCONV;
    }
    q->a = a; q->b = b; q->c = c; q->shortcut = false; q->iters = it;
    return PE_OK;
}

// Eq. deg3_solution: p(x) = beta p_NS(alpha x); also returns beta = max p.
void minimax_cubic(double lo, double hi, double* a, double* b, double* beta) {
    const double alpha = std::sqrt(3.0 / (hi * hi + lo * hi + lo * lo));
    const double alpha3 = cube(alpha);
    const double bt = 4.0 / (2.0 + lo * hi * (lo + hi) * alpha3);
    *a = 1.5 * bt * alpha;
    *b = -0.5 * bt * alpha3;
    *beta = bt;
}

}  // namespace

int coeffs_table(int degree, double l, int T, double safety, double cushion, unsigned flags,
                 double* coeffs, double* bounds, int* remez_iters, const char** why) {
    if (degree != 3 && degree != 5) { *why = "degree must be 3 or 5"; return PE_EINVAL; }
    if (T < 1 || T > kMaxSteps) { *why = "T must be in 1..64"; return PE_EINVAL; }
    if (!(l > 0.0 && l <= 1.0)) { *why = "l must satisfy 0 < l <= 1"; return PE_EINVAL; }
    if (!(safety >= 1.0) || !std::isfinite(safety)) { *why = "safety must be >= 1"; return PE_EINVAL; }
    if (!coeffs) { *why = "coeffs is NULL"; return PE_EINVAL; }
    if (cushion < 0.0) cushion = (degree == 5) ? kKappa5 : kKappa3;
    if (!(cushion <= 1.0)) { *why = "cushion must be <= 1"; return PE_EINVAL; }

    double raw[kMaxSteps][3];
    bool sc[kMaxSteps];
    double u = 1.0;
    if (bounds) { bounds[0] = l; bounds[1] = u; }
    for (int t = 0; t < T; ++t) {
        const double ku = cushion * u;
        const double lo = (l > ku) ? l : ku;   // max(l, kappa u)
        double a, b, c, pmax;
        if (degree == 5) {
            Quintic q;
            int st = minimax_quintic(lo, u, &q);
            if (st != PE_OK) { *why = "Remez iteration did not converge"; return st; }
            a = q.a; b = q.b; c = q.c;
            sc[t] = q.shortcut;
            if (remez_iters) remez_iters[t] = q.iters;
            pmax = odd5(a, b, c, u);      // quintic alternation ends on a max at u
        } else {
            if (!(lo > 0.0 && u > 0.0)) { *why = "degenerate interval"; return PE_EINVAL; }
            double beta;
            minimax_cubic(lo, u, &a, &b, &beta);
            c = 0.0;
            sc[t] = (lo / u >= kShortcut);
            if (remez_iters) remez_iters[t] = 0;
            pmax = beta;                  // cubic's max is its interior extremum
        }
        const double pl = odd5(a, b, c, l);
        const double r = 2.0 / (pl + pmax);
        a = a * r; b = b * r; c = c * r;
        raw[t][0] = a; raw[t][1] = b; raw[t][2] = c;
        l = odd5(a, b, c, l);
        u = 2.0 - l;
        if (bounds) { bounds[2 * (t + 1)] = l; bounds[2 * (t + 1) + 1] = u; }
    }
    const double s3 = safety * safety * safety;
    const double s5 = s3 * safety * safety;
    for (int t = 0; t < T; ++t) {
        const bool skip = sc[t] || safety == 1.0 ||
                          ((flags & PE_SAFETY_SKIP_LAST) && t == T - 1);
        if (skip) {
            coeffs[3 * t + 0] = raw[t][0];
            coeffs[3 * t + 1] = raw[t][1];
            coeffs[3 * t + 2] = raw[t][2];
        } else {
            coeffs[3 * t + 0] = raw[t][0] / safety;
            coeffs[3 * t + 1] = raw[t][1] / s3;
            coeffs[3 * t + 2] = raw[t][2] / s5;
        }
    }
    return PE_OK;
}

}  // namespace pe
