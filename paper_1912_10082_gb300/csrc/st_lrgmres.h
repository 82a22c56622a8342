// Low-rank flexible GMRES (LR-FGMRES), the comparison solver of Section 5,
// Example 1 (Table 1): GMRES on B vec(U) = vec(F) for the matrix form
// L(U) = M U D_t^T + A U C_t^T (Section 4) with every Krylov vector held as
// low-rank factors, right-preconditioned by a nonlinear map (a fixed number
// of RKSM steps), hence the flexible variant.
//
// This header is the method's host driver only: the Arnoldi process over
// vectors that a Backend stores and combines, the Hessenberg least squares by
// Givens rotations, the stopping rule and the memory count.  Where the
// factors live (host or device), how sums are truncated and what the
// preconditioner is belong to the Backend.  Host-only C++ (no CUDA).
//
// Steps, with X_0 = 0 and no restart: V_1 = F / beta (beta = ||F||_F);
// step j: Z_j = P(V_j), W = L(Z_j), classical Gram-Schmidt of W against
// V_1..V_j run twice, h_{j+1,j} = ||W||_F, V_{j+1} = W / h_{j+1,j}; the
// Givens-reduced least-squares residual |g_{j+1}| / beta is the estimate the
// iteration stops on (<= tol, or an exact breakdown h_{j+1,j} = 0 with a
// nonsingular rotated diagonal; a vanishing rotated diagonal is reported as
// stagnation, converged = false, without step j); then
// X = sum_i Z_i y_i with R y = g.  mu_mem counts the stored columns of
// V_1..V_{m+1} and Z_1..Z_m.
#pragma once

#include <cmath>
#include <vector>

namespace lrgmres {

// Storage and arithmetic of the low-rank vectors, addressed by integer ids
// that the driver chooses (0 .. 2 maxit + 4).  Every call returns 0 or a
// negative status, which the driver passes on.
struct Backend {
    virtual ~Backend() = default;
    virtual int inner(int a, int b, double* out) = 0;                   // trace(X_a^T X_b)
    virtual int combine(int dst, const double* c, const int* src, int n) = 0;   // X_dst = trunc(sum c_i X_src_i); dst not in src
    virtual int apply(int dst, int src) = 0;                            // X_dst = trunc(L(X_src))
    virtual int precondition(int dst, int src) = 0;                     // X_dst = P(X_src)
    virtual int rank(int id) const = 0;                                 // columns of X_id's factors
};

// Host half of the truncation of X = P Q^T (reading of the oracle's step 2):
// given R_P (r x r, upper) from a QR P = Q_P R_P computed where P lives, and
// Q (n_t x r) on the host, factor Q = Q_Q R_Q with q = min(r, n_t) columns
// (Householder when r <= n_t; otherwise Q_Q = I and R_Q = Q, n_t x r), take
// the SVD R_P R_Q^T = U S V^T (r x q) and keep the k singular
// values above trunc * largest.  Outputs: Cp (r x k, ld r) with
// P' = Q_P Cp = Q_P U_k S_k, and Qn (n_t x k, ld n_t) = Q_Q V_k, so that
// P' Qn^T is the truncation of X.  svd(m, n, A, lda, U, s, Vt) is a one-sided
// SVD of an m x n matrix, m >= n (the library's dense::svd_small);
// qr(m, n, A, lda, R, ldr) a thin QR with A <- Q (dense::thin_qr).
template <class Svd, class Qr>
inline int truncate_core(int r, const double* RP, int ldrp, int nt, const double* Q, int ldq, double trunc, Svd svd,
                         Qr qr, std::vector<double>* Cp, std::vector<double>* Qn, int* k) {
    *k = 0;
    Cp->clear();
    Qn->clear();
    if (r == 0 || nt == 0) return 0;
    const int q = r <= nt ? r : nt;
    std::vector<double> QQ((size_t)nt * q, 0.0), RQ((size_t)q * r, 0.0);   // Q = QQ RQ, RQ q x r (ld q)
    if (r <= nt) {
        for (int c = 0; c < r; ++c)
            for (int i = 0; i < nt; ++i) QQ[(size_t)c * nt + i] = Q[(size_t)c * ldq + i];
        qr(nt, r, QQ.data(), nt, RQ.data(), q);
    } else {
        for (int i = 0; i < nt; ++i) QQ[(size_t)i * nt + i] = 1.0;
        for (int c = 0; c < r; ++c)
            for (int i = 0; i < nt; ++i) RQ[(size_t)c * q + i] = Q[(size_t)c * ldq + i];
    }
    // core K = R_P R_Q^T (r x q)
    std::vector<double> K((size_t)r * q, 0.0);
    for (int j = 0; j < q; ++j)
        for (int i = 0; i < r; ++i) {
            double acc = 0.0;
            for (int t = 0; t < r; ++t) acc += RP[(size_t)t * ldrp + i] * RQ[(size_t)t * q + j];
            K[(size_t)j * r + i] = acc;
        }
    std::vector<double> U((size_t)r * q), sv(q), Vt((size_t)q * q);
    svd(r, q, K.data(), r, U.data(), sv.data(), Vt.data());
    int kk = 0;
    if (sv[0] > 0.0)
        for (int i = 0; i < q; ++i) kk += sv[i] > trunc * sv[0];
    Cp->assign((size_t)r * kk, 0.0);
    Qn->assign((size_t)nt * kk, 0.0);
    for (int c = 0; c < kk; ++c) {
        for (int i = 0; i < r; ++i) (*Cp)[(size_t)c * r + i] = U[(size_t)c * r + i] * sv[c];
        for (int i = 0; i < nt; ++i) {
            double acc = 0.0;
            for (int t = 0; t < q; ++t) acc += QQ[(size_t)t * nt + i] * Vt[(size_t)t * q + c];
            (*Qn)[(size_t)c * nt + i] = acc;
        }
    }
    *k = kk;
    return 0;
}

struct Options {
    double tol = 1e-8;
    int maxit = 50;
};

struct Result {
    int iterations = 0;
    bool converged = false;
    int mu_mem = 0;
    std::vector<double> history;   // relative residual estimates, history[0] = 1
};

// Ids used by run(): the right-hand side at rhs, the solution written to x;
// V_j at vbase + j, Z_j at zbase + j, two scratch ids for W.
inline int run(Backend& b, int rhs, int x, const Options& o, Result* res) {
    const int maxit = o.maxit > 0 ? o.maxit : 1;
    const int vbase = 2, zbase = vbase + maxit + 1, w0 = zbase + maxit, w1 = w0 + 1;
    if (rhs == x || (rhs >= vbase && rhs <= w1) || (x >= vbase && x <= w1)) return -1;
    Result r;
    double bb = 0.0;
    int st = b.inner(rhs, rhs, &bb);
    if (st) return st;
    const double beta = std::sqrt(bb > 0.0 ? bb : 0.0);
    r.history.push_back(1.0);
    if (!(beta > 0.0)) {
        if (!(bb == 0.0)) return -1;   // NaN
        st = b.combine(x, nullptr, nullptr, 0);
        if (st) return st;
        r.converged = true;
        r.history.back() = 0.0;
        *res = r;
        return 0;
    }
    const double inv = 1.0 / beta;
    if ((st = b.combine(vbase, &inv, &rhs, 1))) return st;
    // H (maxit + 1) x maxit column-major; Givens rotations; g the rotated beta e_1
    std::vector<double> H((size_t)(maxit + 1) * maxit, 0.0), cs(maxit, 0.0), sn(maxit, 0.0), g(maxit + 1, 0.0);
    g[0] = beta;
    auto h = [&](int i, int j) -> double& { return H[(size_t)j * (maxit + 1) + i]; };
    int m = 0, wcur = w0;
    for (int j = 0; j < maxit; ++j) {
        if ((st = b.precondition(zbase + j, vbase + j))) return st;
        if ((st = b.apply(wcur, zbase + j))) return st;
        std::vector<double> coef(j + 2);
        std::vector<int> src(j + 2);
        for (int pass = 0; pass < 2; ++pass) {   // classical Gram-Schmidt, twice
            coef[0] = 1.0;
            src[0] = wcur;
            for (int i = 0; i <= j; ++i) {
                double hij = 0.0;
                if ((st = b.inner(vbase + i, wcur, &hij))) return st;
                h(i, j) += hij;
                coef[i + 1] = -hij;
                src[i + 1] = vbase + i;
            }
            const int wnext = wcur == w0 ? w1 : w0;
            if ((st = b.combine(wnext, coef.data(), src.data(), j + 2))) return st;
            wcur = wnext;
        }
        double ww = 0.0;
        if ((st = b.inner(wcur, wcur, &ww))) return st;
        const double hn = std::sqrt(ww > 0.0 ? ww : 0.0);
        h(j + 1, j) = hn;
        // apply the earlier rotations to column j, then zero its subdiagonal
        for (int i = 0; i < j; ++i) {
            const double a = h(i, j), c = h(i + 1, j);
            h(i, j) = cs[i] * a + sn[i] * c;
            h(i + 1, j) = -sn[i] * a + cs[i] * c;
        }
        const double a = h(j, j), c = h(j + 1, j);
        const double rr = std::hypot(a, c);
        if (!(rr > 0.0)) {
            // h(j,j) and h(j+1,j) both vanish after the rotations: the new preconditioned
            // direction adds nothing (L Z_j lies in span V_1..V_j, e.g. a preconditioner
            // output truncated to rank 0), so the least-squares matrix is singular at this
            // step.  That is stagnation, not convergence: the estimate stays |g_j| / beta
            // and step j does not enter the solution.
            r.history.push_back(std::fabs(g[j]) / beta);
            r.converged = false;
            break;
        }
        cs[j] = a / rr;
        sn[j] = c / rr;
        h(j, j) = rr;
        h(j + 1, j) = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        const double est = std::fabs(g[j + 1]) / beta;
        r.history.push_back(est);
        m = j + 1;
        if (est <= o.tol || hn == 0.0) {
            // hn == 0 with rr > 0 is the exact (lucky) breakdown: g_{j+1} = 0 and R is nonsingular
            r.converged = true;
            break;
        }
        if (j + 1 < maxit) {
            const double ih = 1.0 / hn;
            if ((st = b.combine(vbase + j + 1, &ih, &wcur, 1))) return st;
        }
    }
    // R y = g (upper triangular, m x m)
    std::vector<double> y(m, 0.0);
    for (int i = m - 1; i >= 0; --i) {
        double s = g[i];
        for (int k = i + 1; k < m; ++k) s -= h(i, k) * y[k];
        y[i] = h(i, i) != 0.0 ? s / h(i, i) : 0.0;
    }
    std::vector<int> zs(m);
    for (int i = 0; i < m; ++i) zs[i] = zbase + i;
    if ((st = b.combine(x, y.data(), zs.data(), m))) return st;
    r.iterations = m;
    r.mu_mem = b.rank(wcur);
    for (int i = 0; i < m; ++i) r.mu_mem += b.rank(vbase + i) + b.rank(zbase + i);
    *res = r;
    return 0;
}

}  // namespace lrgmres
