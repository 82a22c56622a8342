// The LR-FGMRES host driver (csrc/st_lrgmres.h) with a dense host backend, on
// the CPU.  Reads a problem written by tests/test_lrgmres_driver.py
// ("n_h n_t p", then M, A (n_h x n_h), D, C (n_t x n_t), F1 (n_h x p),
// F2 (n_t x p), column-major), runs the driver with the identity or the exact
// preconditioner, and prints the residual history, the iteration count, mu_mem
// and the dense solution for comparison with the oracle.
//
// usage: lrgmres_check <file> <identity|exact> <maxit> <tol> <trunc>
//        lrgmres_check <file> truncate <trunc>   (file: "n_h n_t r", P, Q; prints k and P' Q'^T)
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "st_common.cuh"
#include "st_lrgmres.h"

namespace {

struct Factors {
    int r = 0;
    std::vector<double> P, Q;   // n_h x r and n_t x r, column-major
};

class DenseBackend : public lrgmres::Backend {
public:
    DenseBackend(int nh, int nt, std::vector<double> M, std::vector<double> A, std::vector<double> D,
                 std::vector<double> C, double trunc, bool exact)
        : nh_(nh), nt_(nt), M_(std::move(M)), A_(std::move(A)), D_(std::move(D)), C_(std::move(C)), trunc_(trunc),
          exact_(exact) {
        if (exact_) {
            // B = D (x) M + C (x) A, row (l, j) = l n_h + j, column (k, i) = k n_h + i
            const int N = nh_ * nt_;
            B_.assign((size_t)N * N, 0.0);
            for (int k = 0; k < nt_; ++k)
                for (int i = 0; i < nh_; ++i)
                    for (int l = 0; l < nt_; ++l)
                        for (int j = 0; j < nh_; ++j)
                            B_[(size_t)(k * nh_ + i) * N + l * nh_ + j] =
                                D_[(size_t)k * nt_ + l] * M_[(size_t)i * nh_ + j] +
                                C_[(size_t)k * nt_ + l] * A_[(size_t)i * nh_ + j];
            piv_.resize(N);
            ok_ = dense::lu(N, B_.data(), N, piv_.data());
        }
    }
    Factors& at(int id) { return v_[id]; }

    int inner(int a, int b, double* out) override {
        const Factors &x = v_[a], &y = v_[b];
        double s = 0.0;
        for (int k = 0; k < x.r; ++k)
            for (int l = 0; l < y.r; ++l) {
                double pp = 0.0, qq = 0.0;
                for (int i = 0; i < nh_; ++i) pp += x.P[(size_t)k * nh_ + i] * y.P[(size_t)l * nh_ + i];
                for (int i = 0; i < nt_; ++i) qq += x.Q[(size_t)k * nt_ + i] * y.Q[(size_t)l * nt_ + i];
                s += pp * qq;
            }
        *out = s;
        return 0;
    }
    int combine(int dst, const double* c, const int* src, int n) override {
        std::vector<double> X((size_t)nh_ * nt_, 0.0);
        for (int t = 0; t < n; ++t) {
            const Factors& f = v_[src[t]];
            add_dense(f, c[t], X);
        }
        truncate(X, v_[dst]);
        return 0;
    }
    int apply(int dst, int src) override {
        // L(X) = M X D^T + A X C^T, formed densely
        std::vector<double> X((size_t)nh_ * nt_, 0.0), Y((size_t)nh_ * nt_, 0.0);
        add_dense(v_[src], 1.0, X);
        for (int l = 0; l < nt_; ++l)
            for (int j = 0; j < nh_; ++j) {
                double s = 0.0;
                for (int k = 0; k < nt_; ++k) {
                    const double dlk = D_[(size_t)k * nt_ + l], clk = C_[(size_t)k * nt_ + l];
                    if (dlk == 0.0 && clk == 0.0) continue;
                    double mx = 0.0, ax = 0.0;
                    for (int i = 0; i < nh_; ++i) {
                        mx += M_[(size_t)i * nh_ + j] * X[(size_t)k * nh_ + i];
                        ax += A_[(size_t)i * nh_ + j] * X[(size_t)k * nh_ + i];
                    }
                    s += dlk * mx + clk * ax;
                }
                Y[(size_t)l * nh_ + j] = s;
            }
        truncate(Y, v_[dst]);
        return 0;
    }
    int precondition(int dst, int src) override {
        if (zero_) {   // a preconditioner whose output truncates to rank 0
            v_[dst] = Factors{};
            v_[dst].r = 0;
            return 0;
        }
        if (!exact_) {
            v_[dst] = v_[src];
            return 0;
        }
        if (!ok_) return -4;
        std::vector<double> X((size_t)nh_ * nt_, 0.0);
        add_dense(v_[src], 1.0, X);
        const int N = nh_ * nt_;
        dense::lu_solve(N, B_.data(), N, piv_.data(), X.data(), N, 1);
        truncate(X, v_[dst]);
        return 0;
    }
    void set_zero_preconditioner(bool z) { zero_ = z; }
    int rank(int id) const override {
        auto it = v_.find(id);
        return it == v_.end() ? 0 : it->second.r;
    }

private:
    void add_dense(const Factors& f, double c, std::vector<double>& X) const {
        for (int k = 0; k < f.r; ++k)
            for (int l = 0; l < nt_; ++l) {
                const double q = c * f.Q[(size_t)k * nt_ + l];
                if (q == 0.0) continue;
                for (int i = 0; i < nh_; ++i) X[(size_t)l * nh_ + i] += f.P[(size_t)k * nh_ + i] * q;
            }
    }
    // best approximation of X keeping singular values above trunc * largest
    void truncate(const std::vector<double>& X, Factors& out) const {
        const bool tall = nh_ >= nt_;
        const int m = tall ? nh_ : nt_, n = tall ? nt_ : nh_;
        std::vector<double> S((size_t)m * n);
        for (int c = 0; c < n; ++c)
            for (int r = 0; r < m; ++r) S[(size_t)c * m + r] = tall ? X[(size_t)c * nh_ + r] : X[(size_t)r * nh_ + c];
        std::vector<double> U((size_t)m * n), s(n), Vt((size_t)n * n);
        dense::svd_small(m, n, S.data(), m, U.data(), s.data(), Vt.data());
        int r = 0;
        if (n > 0 && s[0] > 0.0)
            for (int k = 0; k < n; ++k) r += s[k] > trunc_ * s[0];
        out.r = r;
        out.P.assign((size_t)nh_ * r, 0.0);
        out.Q.assign((size_t)nt_ * r, 0.0);
        for (int k = 0; k < r; ++k) {
            // tall: X = U S Vt, P = U_k s_k, Q = Vt row k; wide: X^T = U S Vt, P = Vt row k s_k, Q = U_k
            for (int i = 0; i < nh_; ++i)
                out.P[(size_t)k * nh_ + i] = tall ? U[(size_t)k * m + i] * s[k] : Vt[(size_t)i * n + k] * s[k];
            for (int i = 0; i < nt_; ++i)
                out.Q[(size_t)k * nt_ + i] = tall ? Vt[(size_t)i * n + k] : U[(size_t)k * m + i];
        }
    }

    int nh_, nt_;
    std::vector<double> M_, A_, D_, C_, B_;
    std::vector<int> piv_;
    bool ok_ = true;
    double trunc_;
    bool exact_;
    bool zero_ = false;
    std::map<int, Factors> v_;
};

std::vector<double> read(FILE* f, size_t n) {
    std::vector<double> x(n);
    for (auto& v : x)
        if (std::fscanf(f, "%lf", &v) != 1) std::exit(2);
    return x;
}

}  // namespace

// The host half of the truncation (lrgmres::truncate_core), with R_P from a
// Householder QR of P standing in for the device block QR.
int truncate_mode(const char* path, double trunc) {
    FILE* f = std::fopen(path, "r");
    if (!f) return 2;
    int nh, nt, r;
    if (std::fscanf(f, "%d %d %d", &nh, &nt, &r) != 3) return 2;
    auto P = read(f, (size_t)nh * r), Q = read(f, (size_t)nt * r);
    std::fclose(f);
    std::vector<double> QP = P, RP((size_t)r * r);
    dense::thin_qr(nh, r, QP.data(), nh, RP.data(), r);
    std::vector<double> Cp, Qn;
    int k = 0;
    const int st = lrgmres::truncate_core(r, RP.data(), r, nt, Q.data(), nt, trunc, dense::svd_small,
                                          dense::thin_qr, &Cp, &Qn, &k);
    std::printf("status %d\nk %d\nX", st, k);
    for (int l = 0; l < nt; ++l)
        for (int i = 0; i < nh; ++i) {
            double acc = 0.0;
            for (int c = 0; c < k; ++c) {
                double pc = 0.0;
                for (int t = 0; t < r; ++t) pc += QP[(size_t)t * nh + i] * Cp[(size_t)c * r + t];
                acc += pc * Qn[(size_t)c * nt + l];
            }
            std::printf(" %.17g", acc);
        }
    std::printf("\n");
    return st == 0 ? 0 : 1;
}

int main(int argc, char** argv) {
    if (argc == 4 && std::string(argv[2]) == "truncate") return truncate_mode(argv[1], std::atof(argv[3]));
    if (argc != 6) return 2;
    FILE* f = std::fopen(argv[1], "r");
    if (!f) return 2;
    int nh, nt, p;
    if (std::fscanf(f, "%d %d %d", &nh, &nt, &p) != 3) return 2;
    auto M = read(f, (size_t)nh * nh), A = read(f, (size_t)nh * nh);
    auto D = read(f, (size_t)nt * nt), C = read(f, (size_t)nt * nt);
    auto F1 = read(f, (size_t)nh * p), F2 = read(f, (size_t)nt * p);
    std::fclose(f);
    const bool exact = std::string(argv[2]) == "exact";
    lrgmres::Options o;
    o.maxit = std::atoi(argv[3]);
    o.tol = std::atof(argv[4]);
    DenseBackend b(nh, nt, M, A, D, C, std::atof(argv[5]), exact);
    b.set_zero_preconditioner(std::string(argv[2]) == "zero");
    Factors& rhs = b.at(0);
    rhs.r = p;
    rhs.P = F1;
    rhs.Q = F2;
    lrgmres::Result r;
    const int x = 1;
    const int st = lrgmres::run(b, 0, x, o, &r);
    std::printf("status %d\nits %d\nconverged %d\nmu %d\nhist", st, r.iterations, (int)r.converged, r.mu_mem);
    for (double h : r.history) std::printf(" %.17g", h);
    std::printf("\nX");
    std::vector<double> X((size_t)nh * nt, 0.0);
    const Factors& xf = b.at(x);
    for (int k = 0; k < xf.r; ++k)
        for (int l = 0; l < nt; ++l)
            for (int i = 0; i < nh; ++i) X[(size_t)l * nh + i] += xf.P[(size_t)k * nh + i] * xf.Q[(size_t)k * nt + l];
    for (double v : X) std::printf(" %.17g", v);
    std::printf("\n");
    return st == 0 ? 0 : 1;
}
