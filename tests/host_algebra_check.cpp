// Host dense algebra of the solver (st_dense.cpp): results must not depend on
// the number of host threads, and must solve what they claim to.  Built and
// run by tests/test_host_algebra.py; prints one line per check and the
// eigenvalues of a fixed matrix for comparison with numpy.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include "st_common.cuh"

namespace {

std::vector<double> spd(int n, unsigned seed) {
    std::mt19937 g(seed);
    std::normal_distribution<double> nd;
    std::vector<double> B((size_t)n * n), A((size_t)n * n);
    for (auto& x : B) x = nd(g);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double s = 0;
            for (int k = 0; k < n; ++k) s += B[(size_t)k * n + i] * B[(size_t)k * n + j];
            A[(size_t)j * n + i] = s + (i == j ? n : 0.0);
        }
    return A;
}

// run f with the host treated as busy (one thread per call) or idle (up to 8)
template <class F>
void with_threads(bool one, F f) {
    std::vector<hostpar::ActiveSolve*> hold;
    if (one)
        for (int q = 0; q < 4096; ++q) hold.push_back(new hostpar::ActiveSolve());
    f();
    for (auto* h : hold) delete h;
}

}  // namespace

int main() {
    int bad = 0;
    for (int n : {7, 64, 301, 552}) {
        const std::vector<double> A = spd(n, 3 + n);
        std::vector<double> L1 = A, L8 = A, R1(A), R8(A), E1 = A, E8 = A, w1(n), w8(n);
        bool ok1 = false, ok8 = false;
        with_threads(true, [&] {
            ok1 = dense::cholesky(n, L1.data(), n);
            dense::chol_solve(n, L1.data(), n, R1.data(), n, n);
            dense::sym_eigvals(n, E1.data(), n, w1.data());
        });
        with_threads(false, [&] {
            ok8 = dense::cholesky(n, L8.data(), n);
            dense::chol_solve(n, L8.data(), n, R8.data(), n, n);
            dense::sym_eigvals(n, E8.data(), n, w8.data());
        });
        const bool same = ok1 && ok8 && !std::memcmp(L1.data(), L8.data(), sizeof(double) * L1.size()) &&
                          !std::memcmp(R1.data(), R8.data(), sizeof(double) * R1.size()) &&
                          !std::memcmp(w1.data(), w8.data(), sizeof(double) * n);
        // L L^T = A and A X = A (X = I) up to rounding
        double e1 = 0, e2 = 0, na = 0;
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                double s = 0;
                for (int k = 0; k <= std::min(i, j); ++k) s += L8[(size_t)k * n + i] * L8[(size_t)k * n + j];
                e1 = std::max(e1, std::fabs(s - A[(size_t)j * n + i]));
                e2 = std::max(e2, std::fabs(R8[(size_t)j * n + i] - (i == j ? 1.0 : 0.0)));
                na = std::max(na, std::fabs(A[(size_t)j * n + i]));
            }
        const bool acc = e1 <= 1e-12 * na * n && e2 <= 1e-10;
        std::printf("n=%d threads=%d same=%d chol_err=%.2e solve_err=%.2e\n", n,
                    hostpar::threads_for((double)n * n * n / 3.0), (int)same, e1 / na, e2);
        bad += !(same && acc);
    }
    // LU with partial pivoting (the convection-diffusion projected recurrence, and the block upper
    // Hessenberg matrix of the residual formula: lower bandwidth 4): A X = B and A^T X = B; the banded
    // matrices also against an LU whose row loops run over every row (the same factors, value for value)
    for (int band : {-1, 4}) for (int n : {7, 64, 301}) {
        std::mt19937 g(100 + n);
        std::normal_distribution<double> nd;
        std::vector<double> A((size_t)n * n), B((size_t)n * 3);
        for (auto& x : A) x = nd(g);
        for (auto& x : B) x = nd(g);
        if (band >= 0)
            for (int j = 0; j < n; ++j)
                for (int i = j + band + 1; i < n; ++i) A[(size_t)j * n + i] = 0.0;
        std::vector<double> F = A, X = B, Xt = B;
        std::vector<int> piv(n);
        const bool ok = dense::lu(n, F.data(), n, piv.data());
        if (band >= 0) {
            std::vector<double> G = A;
            std::vector<int> pg(n);
            for (int j = 0; j < n; ++j) {
                int pr = j;
                for (int i = j + 1; i < n; ++i)
                    if (std::fabs(G[(size_t)j * n + i]) > std::fabs(G[(size_t)j * n + pr])) pr = i;
                pg[j] = pr;
                for (int c = 0; c < n; ++c) std::swap(G[(size_t)c * n + j], G[(size_t)c * n + pr]);
                for (int i = j + 1; i < n; ++i) G[(size_t)j * n + i] /= G[(size_t)j * n + j];
                for (int c = j + 1; c < n; ++c)
                    for (int i = j + 1; i < n; ++i) G[(size_t)c * n + i] -= G[(size_t)j * n + i] * G[(size_t)c * n + j];
            }
            bool same = pg == piv;
            for (size_t q = 0; q < G.size(); ++q) same = same && G[q] == F[q];
            std::printf("lu band=%d n=%d same_as_full=%d\n", band, n, (int)same);
            bad += !same;
        }
        dense::lu_solve(n, F.data(), n, piv.data(), X.data(), n, 3);
        const bool okt = dense::lu_solve_transpose(n, F.data(), n, piv.data(), Xt.data(), n, 3);
        double r = 0, rt = 0, na = 0, nx = 0, nxt = 0;
        for (int c = 0; c < 3; ++c)
            for (int i = 0; i < n; ++i) {
                double s1 = 0, s2 = 0;
                for (int k = 0; k < n; ++k) {
                    s1 += A[(size_t)k * n + i] * X[(size_t)c * n + k];
                    s2 += A[(size_t)i * n + k] * Xt[(size_t)c * n + k];
                }
                r = std::max(r, std::fabs(s1 - B[(size_t)c * n + i]));
                rt = std::max(rt, std::fabs(s2 - B[(size_t)c * n + i]));
                nx = std::max(nx, std::fabs(X[(size_t)c * n + i]));
                nxt = std::max(nxt, std::fabs(Xt[(size_t)c * n + i]));
            }
        for (double x : A) na = std::max(na, std::fabs(x));
        const bool acc = ok && okt && r <= 1e-13 * n * na * nx && rt <= 1e-13 * n * na * nxt;
        std::printf("lu band=%d n=%d resid=%.2e resid_T=%.2e %s\n", band, n, r / (na * nx), rt / (na * nxt),
                    acc ? "ok" : "BAD");
        bad += !acc;
    }
    {
        // a zero column: no pivot, reported
        const int n = 5;
        std::vector<double> A((size_t)n * n, 1.0);
        for (int i = 0; i < n; ++i) A[(size_t)2 * n + i] = 0.0;
        std::vector<int> piv(n);
        const bool singular = !dense::lu(n, A.data(), n, piv.data());
        std::printf("lu singular reported=%d\n", (int)singular);
        bad += !singular;
    }
    // forward substitution on a thread team: bitwise independent of the team, L X = B
    {
        const int n = 400, nr = 24;
        const std::vector<double> S = spd(n, 21);
        std::vector<double> L = S;
        dense::cholesky(n, L.data(), n);
        std::mt19937 g(5);
        std::normal_distribution<double> nd;
        std::vector<double> B((size_t)n * nr);
        for (auto& x : B) x = nd(g);
        std::vector<double> X1 = B, X8 = B;
        with_threads(true, [&] { dense::lower_solve(n, L.data(), n, X1.data(), n, nr); });
        with_threads(false, [&] { dense::lower_solve(n, L.data(), n, X8.data(), n, nr); });
        double r = 0;
        for (int c = 0; c < nr; ++c)
            for (int i = 0; i < n; ++i) {
                double acc = 0;
                for (int k = 0; k <= i; ++k) acc += L[(size_t)k * n + i] * X8[(size_t)c * n + k];
                r = std::max(r, std::fabs(acc - B[(size_t)c * n + i]));
            }
        const bool same = !std::memcmp(X1.data(), X8.data(), sizeof(double) * X1.size());
        std::printf("lower_solve same=%d resid=%.2e\n", (int)same, r);
        bad += !(same && r <= 1e-11);
    }
    // Householder thin QR and symmetric eigenvectors
    {
        const int m = 50, n = 12;
        std::mt19937 g(9);
        std::normal_distribution<double> nd;
        std::vector<double> A((size_t)m * n), Q, R((size_t)n * n);
        for (auto& x : A) x = nd(g);
        Q = A;
        dense::thin_qr(m, n, Q.data(), m, R.data(), n);
        double orth = 0, rec = 0, low = 0;
        for (int a = 0; a < n; ++a)
            for (int b = 0; b < n; ++b) {
                double qq = 0;
                for (int r = 0; r < m; ++r) qq += Q[(size_t)a * m + r] * Q[(size_t)b * m + r];
                orth = std::max(orth, std::fabs(qq - (a == b ? 1.0 : 0.0)));
                if (a > b) low = std::max(low, std::fabs(R[(size_t)b * n + a]));
            }
        for (int c = 0; c < n; ++c)
            for (int r = 0; r < m; ++r) {
                double acc = 0;
                for (int k = 0; k <= c; ++k) acc += Q[(size_t)k * m + r] * R[(size_t)c * n + k];
                rec = std::max(rec, std::fabs(acc - A[(size_t)c * m + r]));
            }
        const int ne = 40;
        const std::vector<double> S = spd(ne, 13);
        std::vector<double> Z = S, w(ne);
        dense::sym_eig(ne, Z.data(), ne, w.data());
        double er = 0, eo = 0, ns = 0;
        for (double x : S) ns = std::max(ns, std::fabs(x));
        for (int c = 0; c < ne; ++c)
            for (int r = 0; r < ne; ++r) {
                double az = 0, zz = 0;
                for (int k = 0; k < ne; ++k) {
                    az += S[(size_t)k * ne + r] * Z[(size_t)c * ne + k];
                    zz += Z[(size_t)r * ne + k] * Z[(size_t)c * ne + k];
                }
                er = std::max(er, std::fabs(az - w[c] * Z[(size_t)c * ne + r]));
                eo = std::max(eo, std::fabs(zz - (r == c ? 1.0 : 0.0)));
            }
        const bool ok = orth <= 1e-14 && rec <= 1e-13 && low == 0.0 && er <= 1e-13 * ns * ne && eo <= 1e-13;
        std::printf("thin_qr orth=%.2e rec=%.2e lower=%.1e sym_eig resid=%.2e orth=%.2e %s\n", orth, rec, low,
                    er / ns, eo, ok ? "ok" : "BAD");
        bad += !ok;
    }
    // thin QR of a wide matrix (a time factor F2 with fewer rows than columns): A = Q R, the first m
    // columns of Q orthonormal, the others zero, R zero from row m on; the arrays are sized exactly and
    // surrounded by guard values that must stay untouched
    {
        const int m = 3, n = 16, guard = 64;
        std::mt19937 g(21);
        std::normal_distribution<double> nd;
        std::vector<double> A((size_t)m * n), Qb((size_t)m * n + 2 * guard, 7.0), Rb((size_t)n * n + 2 * guard, 7.0);
        for (auto& x : A) x = nd(g);
        double* Q = Qb.data() + guard;
        double* R = Rb.data() + guard;
        std::memcpy(Q, A.data(), sizeof(double) * m * n);
        dense::thin_qr(m, n, Q, m, R, n);
        bool guards = true;
        for (int i = 0; i < guard; ++i)
            guards = guards && Qb[i] == 7.0 && Qb[guard + (size_t)m * n + i] == 7.0 && Rb[i] == 7.0 &&
                     Rb[guard + (size_t)n * n + i] == 7.0;
        double orth = 0, rec = 0, zero = 0;
        for (int a = 0; a < n; ++a)
            for (int b = 0; b < n; ++b) {
                double qq = 0;
                for (int r = 0; r < m; ++r) qq += Q[(size_t)a * m + r] * Q[(size_t)b * m + r];
                orth = std::max(orth, std::fabs(qq - (a == b && a < m ? 1.0 : 0.0)));
                if (a >= m || a > b) zero = std::max(zero, std::fabs(R[(size_t)b * n + a]));
            }
        for (int c = 0; c < n; ++c)
            for (int r = 0; r < m; ++r) {
                double acc = 0;
                for (int k = 0; k < n; ++k) acc += Q[(size_t)k * m + r] * R[(size_t)c * n + k];
                rec = std::max(rec, std::fabs(acc - A[(size_t)c * m + r]));
            }
        const bool ok = guards && orth <= 1e-14 && rec <= 1e-13 && zero == 0.0;
        std::printf("thin_qr wide guards=%d orth=%.2e rec=%.2e zero=%.1e %s\n", (int)guards, orth, rec, zero,
                    ok ? "ok" : "BAD");
        bad += !ok;
    }
    // one-sided Jacobi SVD (rank compression of F): graded singular values 1 .. 1e-14 between random
    // orthogonal factors (Householder QR of Gaussian matrices), tall and square
    for (int shape = 0; shape < 2; ++shape) {
        const int sm = shape == 0 ? 15 : 12, sn = 12;
        std::mt19937 g(11 + shape);
        std::normal_distribution<double> nd;
        std::vector<double> Gu((size_t)sm * sn), Gv((size_t)sn * sn), Ru((size_t)sn * sn), Rv((size_t)sn * sn);
        for (auto& x : Gu) x = nd(g);
        for (auto& x : Gv) x = nd(g);
        dense::thin_qr(sm, sn, Gu.data(), sm, Ru.data(), sn);
        dense::thin_qr(sn, sn, Gv.data(), sn, Rv.data(), sn);
        std::vector<double> sig(sn), B((size_t)sm * sn, 0.0);
        for (int k = 0; k < sn; ++k) sig[k] = std::pow(10.0, -14.0 * k / (sn - 1));
        for (int c = 0; c < sn; ++c)
            for (int r = 0; r < sm; ++r) {
                double acc = 0;
                for (int k = 0; k < sn; ++k) acc += Gu[(size_t)k * sm + r] * sig[k] * Gv[(size_t)k * sn + c];
                B[(size_t)c * sm + r] = acc;
            }
        std::vector<double> U((size_t)sm * sn), sv(sn), Vt((size_t)sn * sn);
        dense::svd_small(sm, sn, B.data(), sm, U.data(), sv.data(), Vt.data());
        // reconstruction, orthogonality of V, orthonormality of U's columns with sigma above 1e-8
        double rec = 0, orv = 0, oru = 0;
        for (int c = 0; c < sn; ++c)
            for (int r = 0; r < sm; ++r) {
                double acc = 0;
                for (int k = 0; k < sn; ++k) acc += U[(size_t)k * sm + r] * sv[k] * Vt[(size_t)c * sn + k];
                rec = std::max(rec, std::fabs(acc - B[(size_t)c * sm + r]));
            }
        for (int a = 0; a < sn; ++a)
            for (int b = 0; b < sn; ++b) {
                double vv = 0, uu = 0;
                for (int k = 0; k < sn; ++k) vv += Vt[(size_t)k * sn + a] * Vt[(size_t)k * sn + b];
                for (int r = 0; r < sm; ++r) uu += U[(size_t)a * sm + r] * U[(size_t)b * sm + r];
                orv = std::max(orv, std::fabs(vv - (a == b ? 1.0 : 0.0)));
                if (sv[a] > 1e-8 && sv[b] > 1e-8) oru = std::max(oru, std::fabs(uu - (a == b ? 1.0 : 0.0)));
            }
        const bool ok = rec <= 1e-14 && orv <= 1e-13 && oru <= 1e-7;
        std::printf("svd %dx%d rec=%.2e orthV=%.2e orthU=%.2e %s\n", sm, sn, rec, orv, oru, ok ? "ok" : "BAD");
        bad += !ok;
        std::printf("svdmat%d %d %d", shape, sm, sn);
        for (double x : B) std::printf(" %.17g", x);
        std::printf("\nsvdval%d", shape);
        for (double x : sv) std::printf(" %.17g", x);
        std::printf("\n");
    }
    // eigenvalues of a fixed 40 x 40 matrix for the numpy comparison
    const int m = 40;
    std::vector<double> C = spd(m, 7), w(m);
    std::printf("mat");
    for (double x : C) std::printf(" %.17g", x);
    std::printf("\n");
    dense::sym_eigvals(m, C.data(), m, w.data());
    std::printf("eig");
    for (double x : w) std::printf(" %.17g", x);
    std::printf("\n%s\n", bad ? "FAIL" : "PASS");
    return bad;
}
