// Cubic B-spline matrices of the wave equation's space-time system (paper
// Section 3 "The Wave Equation"; Section 5 Example 2 uses cubic B-splines in
// space and time), assembled on the host.  See st_wave_matrices in st.h.
//
// Basis: the cubic B-splines N_0..N_{n+2} of the open uniform knot vector
// (0,0,0,0, h, 2h, ..., L,L,L,L) on n intervals of (0, L), evaluated by the
// Cox-de Boor recursion; derivatives from the degree-lowering formula
// N_{i,p}' = p N_{i,p-1} / (t_{i+p} - t_i) - p N_{i+1,p-1} / (t_{i+p+1} - t_{i+1})
// (a term with a zero denominator is zero).  Space keeps N_1..N_{n+1} (zero at
// both ends: H^2 cap H^1_0), time keeps N_0..N_n (value and slope zero at T).
// Integrals by 4-point Gauss-Legendre on every knot interval (exact for the
// degree-6 products of cubic pieces).
#include <cmath>
#include <vector>

#include "st.h"

namespace {

struct Basis {
    int n;                  // intervals
    double len;
    std::vector<double> t;  // knots, n + 7 of them
    int count() const { return n + 3; }
};

Basis make_basis(int n, double len) {
    Basis b{n, len, {}};
    for (int q = 0; q < 3; ++q) b.t.push_back(0.0);
    for (int k = 0; k <= n; ++k) b.t.push_back(len * k / n);
    for (int q = 0; q < 3; ++q) b.t.push_back(len);
    return b;
}

inline double ratio(double a, double d) { return d > 0.0 ? a / d : 0.0; }

// values, first and second derivatives of every cubic B-spline at x (x inside (0, len))
void eval(const Basis& b, double x, std::vector<double>& v0, std::vector<double>& v1, std::vector<double>& v2) {
    const std::vector<double>& t = b.t;
    const int m = (int)t.size() - 1;   // degree-0 functions N_{i,0}, i = 0..m-1
    std::vector<std::vector<double>> N(4, std::vector<double>(m, 0.0));
    for (int i = 0; i < m; ++i) N[0][i] = (t[i] <= x && x < t[i + 1]) ? 1.0 : 0.0;
    for (int p = 1; p <= 3; ++p)
        for (int i = 0; i + p < m; ++i)
            N[p][i] = ratio(x - t[i], t[i + p] - t[i]) * N[p - 1][i] +
                      ratio(t[i + p + 1] - x, t[i + p + 1] - t[i + 1]) * N[p - 1][i + 1];
    const int nb = b.count();
    v0.assign(nb, 0.0);
    v1.assign(nb, 0.0);
    v2.assign(nb, 0.0);
    // N_{i,2}' for the second derivatives of the cubics
    std::vector<double> d2(m, 0.0);
    for (int i = 0; i + 2 < m; ++i)
        d2[i] = 2.0 * ratio(N[1][i], t[i + 2] - t[i]) - 2.0 * ratio(N[1][i + 1], t[i + 3] - t[i + 1]);
    for (int i = 0; i < nb; ++i) {
        v0[i] = N[3][i];
        v1[i] = 3.0 * ratio(N[2][i], t[i + 3] - t[i]) - 3.0 * ratio(N[2][i + 1], t[i + 4] - t[i + 1]);
        v2[i] = 3.0 * ratio(d2[i], t[i + 3] - t[i]) - 3.0 * ratio(d2[i + 1], t[i + 4] - t[i + 1]);
    }
}

// G[a][b] = (D^da phi_a, D^db phi_b) for the kept functions first..first+N-1 (column-major, N x N)
void gram(const Basis& b, int first, int N, int da, int db, double* G) {
    if (!G) return;
    for (size_t e = 0; e < (size_t)N * N; ++e) G[e] = 0.0;
    // 4-point Gauss-Legendre on [-1, 1]
    const double s = std::sqrt(6.0 / 5.0);
    const double xa = std::sqrt(3.0 / 7.0 - 2.0 / 7.0 * s), xb = std::sqrt(3.0 / 7.0 + 2.0 / 7.0 * s);
    const double wa = (18.0 + std::sqrt(30.0)) / 36.0, wb = (18.0 - std::sqrt(30.0)) / 36.0;
    const double gx[4] = {-xb, -xa, xa, xb}, gw[4] = {wb, wa, wa, wb};
    std::vector<double> v[3];
    const double h = b.len / b.n;
    for (int k = 0; k < b.n; ++k) {
        const double a0 = b.len * k / b.n;
        for (int q = 0; q < 4; ++q) {
            const double x = a0 + 0.5 * h * (gx[q] + 1.0), w = 0.5 * h * gw[q];
            eval(b, x, v[0], v[1], v[2]);
            // only the 4 cubics nonzero on interval k: indices k..k+3
            for (int i = k; i <= k + 3; ++i) {
                const int r = i - first;
                if (r < 0 || r >= N) continue;
                for (int j = k; j <= k + 3; ++j) {
                    const int c = j - first;
                    if (c < 0 || c >= N) continue;
                    G[(size_t)c * N + r] += w * v[da][i] * v[db][j];
                }
            }
        }
    }
}

}  // namespace

extern "C" int st_wave_matrices(int n_x, int n_t, double T, double* Mh, double* Ah, double* Qh, double* Mt,
                                double* Dt, double* Qt) {
    if (n_x < 4 || n_t < 4 || !(T > 0.0)) return ST_EINVAL;
    const Basis bs = make_basis(n_x, 1.0), bt = make_basis(n_t, T);
    const int Nh = n_x + 1, Nt = n_t + 1;
    gram(bs, 1, Nh, 0, 0, Mh);
    gram(bs, 1, Nh, 1, 1, Ah);
    gram(bs, 1, Nh, 2, 2, Qh);
    gram(bt, 0, Nt, 0, 0, Mt);
    gram(bt, 0, Nt, 2, 0, Dt);   // D_t[k, l] = ((rho^k)'', rho^l): row k, column l
    gram(bt, 0, Nt, 2, 2, Qt);
    return ST_OK;
}
