// Small dense FP64 algebra for the projected problems (k x k, k <= a few
// thousand), run on the host cores next to the GPU.  Column-major storage.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

#include "st_common.cuh"

// ---------------------------------------------------------------------------
// Host threads for the projected problems.  Every parallel loop below gives
// each output element to one thread and keeps the serial order of its sum, so
// results are bitwise the same for any thread count (a solve gives the same
// numbers alone and next to others).
// ---------------------------------------------------------------------------
namespace hostpar {

static std::atomic<int> g_active{0};

ActiveSolve::ActiveSolve() { g_active.fetch_add(1); }
ActiveSolve::~ActiveSolve() { g_active.fetch_sub(1); }

namespace {
thread_local int t_budget = 0;   // 0: no budget set on this thread
}

ThreadBudget::ThreadBudget(int n) : prev(t_budget) { t_budget = std::max(1, n); }
ThreadBudget::~ThreadBudget() { t_budget = prev; }

int threads_for(double flops) {
    static const int hw = std::max(1, (int)std::thread::hardware_concurrency());
    if (flops < 4e6) return 1;
    const int share = t_budget > 0 ? t_budget : std::max(1, hw / std::max(1, g_active.load()));
    return std::max(1, std::min({8, share, (int)(flops / 2e6)}));
}

void Barrier::wait() {
    if (n <= 1) return;
    const unsigned g = gen.load(std::memory_order_acquire);
    if (arrived.fetch_add(1, std::memory_order_acq_rel) + 1 == n) {
        arrived.store(0, std::memory_order_relaxed);
        gen.fetch_add(1, std::memory_order_release);
        return;
    }
    int spins = 0;
    while (gen.load(std::memory_order_acquire) == g)
        if (++spins > 2000) std::this_thread::yield();
}

void run(int T, const std::function<void(int, Barrier&)>& body) {
    Barrier b(std::max(1, T));
    if (T <= 1) {
        body(0, b);
        return;
    }
    std::vector<std::thread> th;
    th.reserve(T - 1);
    for (int t = 1; t < T; ++t) th.emplace_back([&body, &b, t] { body(t, b); });
    body(0, b);
    for (auto& x : th) x.join();
}

Pool::Pool(int threads) {
    for (int t = 1; t < threads; ++t) workers_.emplace_back([this] { work(); });
}

Pool::~Pool() {
    {
        std::lock_guard<std::mutex> lk(mu_);
        stop_ = true;
        ++gen_;
    }
    cv_.notify_all();
    for (auto& w : workers_) w.join();
}

void Pool::work() {
    unsigned seen = 0;
    while (true) {
        const std::function<void(int)>* job;
        int n;
        {
            std::unique_lock<std::mutex> lk(mu_);
            cv_.wait(lk, [&] { return gen_ != seen; });
            seen = gen_;
            if (stop_) return;
            job = job_;
            n = n_;
            ++busy_;   // before taking an item: run() waits for busy_ == 0
        }
        {
            ThreadBudget budget(std::max(1, threads() / std::max(1, n)));
            for (int i = next_.fetch_add(1); job && i < n; i = next_.fetch_add(1)) (*job)(i);
        }
        {
            std::lock_guard<std::mutex> lk(mu_);
            --busy_;
        }
        done_cv_.notify_all();
    }
}

void Pool::run(int n, const std::function<void(int)>& f) {
    if (n <= 0) return;
    ThreadBudget budget(std::max(1, threads() / n));
    if (workers_.empty() || n == 1) {
        for (int i = 0; i < n; ++i) f(i);
        return;
    }
    {
        std::unique_lock<std::mutex> lk(mu_);
        done_cv_.wait(lk, [&] { return busy_ == 0; });   // no worker is still inside an earlier job
        job_ = &f;
        n_ = n;
        next_.store(0);
        ++gen_;
    }
    cv_.notify_all();
    for (int i = next_.fetch_add(1); i < n; i = next_.fetch_add(1)) f(i);
    // every item has been taken; wait for the workers still running theirs
    std::unique_lock<std::mutex> lk(mu_);
    done_cv_.wait(lk, [&] { return busy_ == 0; });
    job_ = nullptr;
}

}  // namespace hostpar

namespace dense {

#define A_(i, j) A[(size_t)(j) * lda + (i)]

// Dot product with four independent partial sums (vectorisable without
// reassociation flags; the summation order is fixed).
static inline double dot(int n, const double* x, const double* y) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int i = 0;
    for (; i + 4 <= n; i += 4) {
        s0 += x[i] * y[i];
        s1 += x[i + 1] * y[i + 1];
        s2 += x[i + 2] * y[i + 2];
        s3 += x[i + 3] * y[i + 3];
    }
    for (; i < n; ++i) s0 += x[i] * y[i];
    return (s0 + s1) + (s2 + s3);
}

// Lower Cholesky factor in place, right-looking: each step scales one column
// and updates the trailing columns with contiguous (vectorisable) loops.
bool cholesky(int n, double* A, int lda) {
    // Blocked right-looking order: thread 0 factors a panel of NB columns (each
    // scaled, then applied to the panel's later columns), then the threads apply
    // the panel's columns, in ascending order, to the trailing columns (dealt
    // cyclically).  Every entry receives its updates in ascending column order,
    // so the factor does not depend on the thread count.
    constexpr int NB = 32;
    const int T = hostpar::threads_for((double)n * n * n / 3.0);
    bool ok = true;
    hostpar::run(T, [&](int t, hostpar::Barrier& bar) {
        for (int jb = 0; jb < n; jb += NB) {
            const int je = std::min(n, jb + NB);
            if (t == 0) {
                for (int j = jb; j < je && ok; ++j) {
                    double* cj = A + (size_t)j * lda;
                    const double s = cj[j];
                    if (!(s > 0.0)) {
                        ok = false;
                        break;
                    }
                    const double d = std::sqrt(s);
                    cj[j] = d;
                    for (int i = j + 1; i < n; ++i) cj[i] /= d;
                    for (int c = j + 1; c < je; ++c) {
                        const double tc = cj[c];
                        if (tc == 0.0) continue;
                        double* cc = A + (size_t)c * lda;
                        for (int i = c; i < n; ++i) cc[i] -= cj[i] * tc;
                    }
                }
            }
            bar.wait();
            if (!ok) return;   // read after the barrier: every thread leaves at the same panel
            for (int c = je + t; c < n; c += T) {
                double* cc = A + (size_t)c * lda;
                for (int j = jb; j < je; ++j) {
                    const double* cj = A + (size_t)j * lda;
                    const double tc = cj[c];
                    if (tc == 0.0) continue;
                    for (int i = c; i < n; ++i) cc[i] -= cj[i] * tc;
                }
            }
            bar.wait();
        }
    });
    if (!ok) return false;
    for (int j = 1; j < n; ++j)
        for (int i = 0; i < j; ++i) A_(i, j) = 0.0;
    return true;
}

// L L^T X = B: forward substitution by columns of L (axpy), back substitution
// with L^T by dot products with columns of L; both contiguous.
static void chol_solve_cols(int n, const double* L, int ldl, double* B, int ldb, int c0, int c1) {
    for (int c = c0; c < c1; ++c) {
        double* b = B + (size_t)c * ldb;
        for (int j = 0; j < n; ++j) {
            const double* lj = L + (size_t)j * ldl;
            double t = b[j] / lj[j];
            b[j] = t;
            if (t == 0.0) continue;
            for (int i = j + 1; i < n; ++i) b[i] -= lj[i] * t;
        }
        for (int i = n - 1; i >= 0; --i) {
            const double* li = L + (size_t)i * ldl;
            b[i] = (b[i] - dot(n - i - 1, li + i + 1, b + i + 1)) / li[i];
        }
    }
}

// right-hand sides split over the threads
void chol_solve(int n, const double* L, int ldl, double* B, int ldb, int nrhs) {
    const int T = std::min(nrhs, hostpar::threads_for(2.0 * n * n * nrhs));
    hostpar::run(T, [&](int t, hostpar::Barrier&) {
        chol_solve_cols(n, L, ldl, B, ldb, (int)((long long)nrhs * t / T), (int)((long long)nrhs * (t + 1) / T));
    });
}

// L X = B for lower triangular L (forward substitution by columns of L).
void lower_solve(int n, const double* L, int ldl, double* B, int ldb, int nrhs) {
    const int T = std::min(nrhs, hostpar::threads_for((double)n * n * nrhs));
    hostpar::run(T, [&](int th, hostpar::Barrier&) {
        const int c0 = (int)((long long)nrhs * th / T), c1 = (int)((long long)nrhs * (th + 1) / T);
        for (int c = c0; c < c1; ++c) {
            double* b = B + (size_t)c * ldb;
            for (int j = 0; j < n; ++j) {
                const double* lj = L + (size_t)j * ldl;
                double t = b[j] / lj[j];
                b[j] = t;
                if (t == 0.0) continue;
                for (int i = j + 1; i < n; ++i) b[i] -= lj[i] * t;
            }
        }
    });
}

bool lu(int n, double* A, int lda, int* piv) {
    // lower bandwidth: rows below it are zero in every column (the block upper Hessenberg matrices of
    // the rational Arnoldi relation have a band of one block).  Partial pivoting picks the pivot within
    // the band and the multipliers stay in it, so restricting the row loops to the band computes the
    // same factors in O(n^2 bw) instead of O(n^3)
    int bw = 0;
    for (int j = 0; j < n; ++j)
        for (int i = n - 1; i > j + bw; --i)
            if (A_(i, j) != 0.0) {
                bw = i - j;
                break;
            }
    bool ok = true;
    for (int j = 0; j < n; ++j) {
        const int iend = std::min(n, j + bw + 1);
        int pr = j;
        double mx = std::fabs(A_(j, j));
        for (int i = j + 1; i < iend; ++i)
            if (std::fabs(A_(i, j)) > mx) {
                mx = std::fabs(A_(i, j));
                pr = i;
            }
        piv[j] = pr;
        if (pr != j)
            for (int c = 0; c < n; ++c) std::swap(A_(j, c), A_(pr, c));
        double d = A_(j, j);
        if (d == 0.0) {
            ok = false;
            continue;
        }
        for (int i = j + 1; i < iend; ++i) A_(i, j) /= d;
        for (int c = j + 1; c < n; ++c) {
            double t = A_(j, c);
            if (t == 0.0) continue;
            double* colc = A + (size_t)c * lda;
            const double* colj = A + (size_t)j * lda;
            for (int i = j + 1; i < iend; ++i) colc[i] -= colj[i] * t;
        }
    }
    return ok;
}

void lu_solve(int n, const double* A, int lda, const int* piv, double* B, int ldb, int nrhs) {
    for (int c = 0; c < nrhs; ++c) {
        double* b = B + (size_t)c * ldb;
        for (int i = 0; i < n; ++i)
            if (piv[i] != i) std::swap(b[i], b[piv[i]]);
        for (int j = 0; j < n; ++j) {
            double t = b[j];
            if (t == 0.0) continue;
            for (int i = j + 1; i < n; ++i) b[i] -= A_(i, j) * t;
        }
        for (int j = n - 1; j >= 0; --j) {
            b[j] /= A_(j, j);
            double t = b[j];
            if (t == 0.0) continue;
            for (int i = 0; i < j; ++i) b[i] -= A_(i, j) * t;
        }
    }
}

// Solve A^T x = b with A = P^T L U from lu(): U^T L^T P x = b.
bool lu_solve_transpose(int n, const double* A, int lda, const int* piv, double* B, int ldb, int nrhs) {
    for (int c = 0; c < nrhs; ++c) {
        double* b = B + (size_t)c * ldb;
        for (int j = 0; j < n; ++j) {   // U^T y = b (lower triangular)
            if (A_(j, j) == 0.0) return false;
            b[j] = (b[j] - dot(j, &A_(0, j), b)) / A_(j, j);
        }
        for (int j = n - 1; j >= 0; --j)   // L^T z = y (unit upper)
            b[j] -= dot(n - j - 1, &A_(j + 1, j), b + j + 1);
        for (int i = n - 1; i >= 0; --i)
            if (piv[i] != i) std::swap(b[i], b[piv[i]]);
    }
    return true;
}

// Householder reduction of a symmetric matrix to tridiagonal form T = Q^T A Q.
// d: diagonal, e: sub-diagonal (e[i] couples i and i+1).  If want_q, A is
// overwritten by Q; otherwise A is destroyed.
// The reduction runs on a thread team.  Every thread forms the reflector and
// the scalars itself (the same serial arithmetic, O(n) a step), p = tau A22 v
// is split by rows and the rank-2 update by columns, each element keeping the
// serial order of its sum; two barriers a step.
static void tridiagonalize(int n, double* A, int lda, double* d, double* e, bool want_q) {
    std::vector<double> p(n);
    std::vector<double> taus(n, 0.0);
    // one thread: with two barriers a step the team ran slower than one core on
    // a 552 x 552 reduction (the steps are memory-bound and short)
    const int T = 1;
    hostpar::run(T, [&](int t, hostpar::Barrier& bar) {
        std::vector<double> v(n), w(n);
        for (int j = 0; j + 2 < n; ++j) {
            const int m = n - j - 1;
            double* x = &A_(j + 1, j);
            double alpha = 0.0;
            for (int i = 0; i < m; ++i) alpha += x[i] * x[i];
            alpha = std::sqrt(alpha);
            if (alpha == 0.0) {
                if (t == 0) taus[j] = 0.0;
                continue;   // the same decision in every thread
            }
            if (x[0] > 0) alpha = -alpha;
            // v = x - alpha e1, normalised so that v[0] = 1
            const double v0 = x[0] - alpha;
            for (int i = 0; i < m; ++i) v[i] = x[i] / v0;
            v[0] = 1.0;
            double vv = 0.0;
            for (int i = 0; i < m; ++i) vv += v[i] * v[i];
            const double tau = 2.0 / vv;
            // p = tau * A22 v (symmetric, full storage), by columns of A22, rows split
            const int i0 = (int)((long long)m * t / T), i1 = (int)((long long)m * (t + 1) / T);
            for (int i = i0; i < i1; ++i) p[i] = 0.0;
            for (int k = 0; k < m; ++k) {
                const double* col = &A_(j + 1, j + 1 + k);
                const double vk = v[k];
                for (int i = i0; i < i1; ++i) p[i] += col[i] * vk;
            }
            for (int i = i0; i < i1; ++i) p[i] *= tau;
            bar.wait();
            double pv = 0.0;
            for (int i = 0; i < m; ++i) pv += p[i] * v[i];
            const double K = 0.5 * tau * pv;
            for (int i = 0; i < m; ++i) w[i] = p[i] - K * v[i];
            for (int c = t; c < m; c += T) {
                double* col = &A_(j + 1, j + 1 + c);
                const double vc = v[c], wc = w[c];
                for (int i = 0; i < m; ++i) col[i] -= v[i] * wc + w[i] * vc;
            }
            bar.wait();   // A22 and p are free again; column j is read by nobody from here on
            if (t == 0) {
                taus[j] = tau;
                // store v below the sub-diagonal for Q accumulation
                x[0] = alpha;
                for (int i = 1; i < m; ++i) x[i] = v[i];
            }
        }
    });
    std::vector<double> v(n);
    for (int i = 0; i < n; ++i) d[i] = A_(i, i);
    for (int i = 0; i + 1 < n; ++i) e[i] = A_(i + 1, i);
    if (!want_q) return;
    // Q = H_0 H_1 ... H_{n-3}; accumulate backwards into identity
    std::vector<double> Q((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
    for (int j = n - 3; j >= 0; --j) {
        if (taus[j] == 0.0) continue;
        int m = n - j - 1;
        v[0] = 1.0;
        for (int i = 1; i < m; ++i) v[i] = A_(j + 1 + i, j);
        for (int c = j + 1; c < n; ++c) {
            double* col = &Q[(size_t)c * n + j + 1];
            double s = 0.0;
            for (int i = 0; i < m; ++i) s += v[i] * col[i];
            s *= taus[j];
            for (int i = 0; i < m; ++i) col[i] -= s * v[i];
        }
    }
    for (int c = 0; c < n; ++c) std::memcpy(&A_(0, c), &Q[(size_t)c * n], sizeof(double) * n);
}

// Eigenvalues (and, with Z, eigenvectors) of a symmetric tridiagonal matrix
// by the implicit QL algorithm with Wilkinson-type shifts, the published
// method of Bowdler, Martin, Reinsch and Wilkinson, "The QR and QL algorithms
// for symmetric matrices" (Numer. Math. 11, 1968; EISPACK tql1/tql2), whose
// steps this routine follows.  Z (n x n, ldz) receives the rotations when
// non-null.
static void tridiag_ql(int n, double* d, double* e, double* Z, int ldz) {
    if (n <= 1) return;
    std::vector<double> ee(n, 0.0);
    for (int i = 0; i + 1 < n; ++i) ee[i] = e[i];
    const double eps = 2.220446049250313e-16;
    for (int l = 0; l < n; ++l) {
        int iter = 0;
        while (true) {
            int m;
            for (m = l; m < n - 1; ++m) {
                double dd = std::fabs(d[m]) + std::fabs(d[m + 1]);
                if (std::fabs(ee[m]) <= eps * dd) break;
            }
            if (m == l) break;
            if (++iter > 60) break;
            double g = (d[l + 1] - d[l]) / (2.0 * ee[l]);
            double r = std::hypot(g, 1.0);
            g = d[m] - d[l] + ee[l] / (g + std::copysign(r, g));
            double s = 1.0, c = 1.0, p = 0.0;
            int i;
            bool early = false;
            for (i = m - 1; i >= l; --i) {
                double f = s * ee[i];
                double b = c * ee[i];
                r = std::hypot(f, g);
                ee[i + 1] = r;
                if (r == 0.0) {
                    d[i + 1] -= p;
                    ee[m] = 0.0;
                    early = true;
                    break;
                }
                s = f / r;
                c = g / r;
                g = d[i + 1] - p;
                r = (d[i] - g) * s + 2.0 * c * b;
                p = s * r;
                d[i + 1] = g + p;
                g = c * r - b;
                if (Z) {
                    double* zi = Z + (size_t)i * ldz;
                    double* zi1 = Z + (size_t)(i + 1) * ldz;
                    for (int k = 0; k < n; ++k) {
                        double t = zi1[k];
                        zi1[k] = s * zi[k] + c * t;
                        zi[k] = c * zi[k] - s * t;
                    }
                }
            }
            if (early) continue;
            d[l] -= p;
            ee[l] = g;
            ee[m] = 0.0;
        }
    }
}

static void sort_eig(int n, double* w, double* Z, int ldz) {
    for (int i = 0; i < n; ++i) {
        int k = i;
        for (int j = i + 1; j < n; ++j)
            if (w[j] < w[k]) k = j;
        if (k != i) {
            std::swap(w[i], w[k]);
            if (Z)
                for (int r = 0; r < n; ++r) std::swap(Z[(size_t)i * ldz + r], Z[(size_t)k * ldz + r]);
        }
    }
}

void sym_eigvals(int n, double* A, int lda, double* w) {
    if (n == 0) return;
    std::vector<double> e(n, 0.0);
    tridiagonalize(n, A, lda, w, e.data(), false);
    tridiag_ql(n, w, e.data(), nullptr, 0);
    sort_eig(n, w, nullptr, 0);
}

void sym_eig(int n, double* A, int lda, double* w) {
    if (n == 0) return;
    std::vector<double> e(n, 0.0);
    tridiagonalize(n, A, lda, w, e.data(), true);
    tridiag_ql(n, w, e.data(), A, lda);
    sort_eig(n, w, A, lda);
}

// Householder QR of an m x n matrix: A <- Q (m x n), R (n x n), A = Q R.  For m < n (more columns
// than rows) the reflectors stop at column m: Q's first m columns are orthonormal and the rest zero,
// R's rows from m on are zero (R upper trapezoidal in its first m rows).
int thin_qr(int m, int n, double* A, int lda, double* R, int ldr) {
    const int kq = std::min(m, n);
    std::vector<double> taus(n, 0.0);
    for (int j = 0; j < kq; ++j) {
        double* x = &A_(j, j);
        int len = m - j;
        double alpha = 0.0;
        for (int i = 0; i < len; ++i) alpha += x[i] * x[i];
        alpha = std::sqrt(alpha);
        if (alpha == 0.0) {
            taus[j] = 0.0;
            continue;
        }
        if (x[0] > 0) alpha = -alpha;
        double v0 = x[0] - alpha;
        for (int i = 1; i < len; ++i) x[i] /= v0;
        double vv = 1.0;
        for (int i = 1; i < len; ++i) vv += x[i] * x[i];
        double tau = 2.0 / vv;
        taus[j] = tau;
        x[0] = alpha;
        for (int c = j + 1; c < n; ++c) {
            double* y = &A_(j, c);
            double s = y[0];
            for (int i = 1; i < len; ++i) s += x[i] * y[i];
            s *= tau;
            y[0] -= s;
            for (int i = 1; i < len; ++i) y[i] -= s * x[i];
        }
    }
    for (int c = 0; c < n; ++c)
        for (int r = 0; r < n; ++r) R[(size_t)c * ldr + r] = r <= c && r < m ? A_(r, c) : 0.0;
    // form Q in place, backwards
    std::vector<double> Q((size_t)m * n, 0.0);
    for (int i = 0; i < kq; ++i) Q[(size_t)i * m + i] = 1.0;
    for (int j = kq - 1; j >= 0; --j) {
        if (taus[j] == 0.0) continue;
        int len = m - j;
        for (int c = j; c < kq; ++c) {
            double* y = &Q[(size_t)c * m + j];
            double s = y[0];
            for (int i = 1; i < len; ++i) s += A_(j + i, j) * y[i];
            s *= taus[j];
            y[0] -= s;
            for (int i = 1; i < len; ++i) y[i] -= s * A_(j + i, j);
        }
    }
    for (int c = 0; c < n; ++c) std::memcpy(&A_(0, c), &Q[(size_t)c * m], sizeof(double) * m);
    return 0;
}

// One-sided Jacobi SVD of a small m x n matrix: A = U diag(s) Vt, s descending.
// U: m x n (ld m), s: n, Vt: n x n (ld n).
void svd_small(int m, int n, const double* A, int lda, double* U, double* s, double* Vt) {
    std::vector<double> W((size_t)m * n), V((size_t)n * n, 0.0);
    for (int c = 0; c < n; ++c)
        for (int r = 0; r < m; ++r) W[(size_t)c * m + r] = A_(r, c);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) {
                double a = 0, b = 0, g = 0;
                for (int r = 0; r < m; ++r) {
                    double wi = W[(size_t)i * m + r], wj = W[(size_t)j * m + r];
                    a += wi * wi;
                    b += wj * wj;
                    g += wi * wj;
                }
                if (std::fabs(g) <= 1e-300 || std::fabs(g) <= 1e-15 * std::sqrt(a * b)) continue;
                off = std::max(off, std::fabs(g) / std::sqrt(a * b));
                double zeta = (b - a) / (2.0 * g);
                double t = std::copysign(1.0, zeta) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
                double c = 1.0 / std::sqrt(1.0 + t * t), sn = c * t;
                for (int r = 0; r < m; ++r) {
                    double wi = W[(size_t)i * m + r], wj = W[(size_t)j * m + r];
                    W[(size_t)i * m + r] = c * wi - sn * wj;
                    W[(size_t)j * m + r] = sn * wi + c * wj;
                }
                for (int r = 0; r < n; ++r) {
                    double vi = V[(size_t)i * n + r], vj = V[(size_t)j * n + r];
                    V[(size_t)i * n + r] = c * vi - sn * vj;
                    V[(size_t)j * n + r] = sn * vi + c * vj;
                }
            }
        if (off < 1e-15) break;
    }
    std::vector<int> order(n);
    std::vector<double> sv(n);
    for (int i = 0; i < n; ++i) {
        double a = 0;
        for (int r = 0; r < m; ++r) a += W[(size_t)i * m + r] * W[(size_t)i * m + r];
        sv[i] = std::sqrt(a);
        order[i] = i;
    }
    std::sort(order.begin(), order.end(), [&](int x, int y) { return sv[x] > sv[y]; });
    for (int k = 0; k < n; ++k) {
        int i = order[k];
        s[k] = sv[i];
        for (int r = 0; r < m; ++r) U[(size_t)k * m + r] = sv[i] > 0 ? W[(size_t)i * m + r] / sv[i] : 0.0;
        for (int r = 0; r < n; ++r) Vt[(size_t)r * n + k] = V[(size_t)i * n + r];
    }
}

#undef A_

}  // namespace dense
