// LR-FGMRES+RKSM on the device (paper Section 5, Example 1, the comparison
// column of Table 1): flexible GMRES on the space-time system in matrix form
// L(U) = M U D_t^T + A U C_t^T = F, every Krylov vector a low-rank pair
// X = P Q^T, right-preconditioned by a fixed number of RKSM iterations (a
// nonlinear map, hence the flexible variant).  The Arnoldi process, the
// Givens least squares and the stopping rule are the host driver of
// st_lrgmres.h; this file is its device backend:
//   - P (N_h x r) lives on the device, Q (N_t x r) on the host;
//   - <X, Y> = trace(X^T Y) = sum (Px^T Py) .* (Qx^T Qy): one device Gram
//     product, the N_t-side product on the host;
//   - L(P Q^T) = [M P, A P] [D_t Q, C_t Q]^T: box-stencil products on the
//     device, the bidiagonal time products on the host;
//   - every sum and operator product is truncated: a column-wise QR of P on
//     the device (classical Gram-Schmidt, each column re-projected until it
//     settles), then the host half (QR of Q, SVD of the small core,
//     st_lrgmres.h truncate_core) and P' = Q_P C_p by one tall-skinny product;
//     a sum with more columns than N_t is first multiplied out to the dense
//     N_h x N_t matrix (one GEMM), whose QR has N_t columns;
//   - the preconditioner is st_solve's RKSM driver stopped after
//     `precond_iters` shifted solves on (P, Q) as the load's factors (blocks of
//     at most 16 columns, their results summed), Z = V Y truncated.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <vector>

#include "st_common.cuh"
#include "st_lrgmres.h"
#include "st_rksm.h"

using namespace rksm;

namespace {

struct LrVec {
    int r = 0;
    double* P = nullptr;   // device, n_h x cap, ld n_h
    int cap = 0;
    std::vector<double> Q;   // host, n_t x r, ld n_t
};

class DeviceBackend : public lrgmres::Backend {
   public:
    DeviceBackend(st_problem* p, double trunc, int precond_iters)
        : p_(p), c_{p, p->stream, p->n_h}, n_(p->n_h), nt_(p->n_t), trunc_(trunc), piters_(precond_iters) {}
    ~DeviceBackend() override {
        for (auto& kv : v_)
            if (kv.second.P) st_free_one(p_, kv.second.P);
        for (double* s : scratch_)
            if (s) st_free_one(p_, s);
    }
    int status() const { return st_; }
    int precond_iterations() const { return pits_; }
    LrVec& at(int id) { return v_[id]; }

    // sets X_id = P Q^T (P device n x r, copied; Q host nt x r)
    int set(int id, const double* P, int ldp, const double* Q, int ldq, int r) {
        LrVec& x = v_[id];
        ST_TRY(reserve(x, r));
        if (r > 0)
            ST_CUDA_TRY(cudaMemcpy2DAsync(x.P, sizeof(double) * n_, P, sizeof(double) * ldp, sizeof(double) * n_, r,
                                          cudaMemcpyDeviceToDevice, c_.s));
        x.r = r;
        x.Q.assign((size_t)nt_ * r, 0.0);
        for (int j = 0; j < r; ++j) std::memcpy(&x.Q[(size_t)j * nt_], Q + (size_t)j * ldq, sizeof(double) * nt_);
        return ST_OK;
    }

    int inner(int a, int b, double* out) override {
        const LrVec &x = v_[a], &y = v_[b];
        *out = 0.0;
        if (x.r == 0 || y.r == 0) return ST_OK;
        std::vector<double> G((size_t)x.r * y.r);
        if (int st = ts_tn_host(c_, x.r, y.r, x.P, n_, y.P, n_, G.data())) return fail(st);
        double s = 0.0;
        for (int j = 0; j < y.r; ++j)
            for (int i = 0; i < x.r; ++i) {
                // four partial sums in a fixed order (vectorisable without reassociation)
                double q0 = 0.0, q1 = 0.0, q2 = 0.0, q3 = 0.0;
                const double* qi = &x.Q[(size_t)i * nt_];
                const double* qj = &y.Q[(size_t)j * nt_];
                int l = 0;
                for (; l + 4 <= nt_; l += 4) {
                    q0 += qi[l] * qj[l];
                    q1 += qi[l + 1] * qj[l + 1];
                    q2 += qi[l + 2] * qj[l + 2];
                    q3 += qi[l + 3] * qj[l + 3];
                }
                for (; l < nt_; ++l) q0 += qi[l] * qj[l];
                s += G[(size_t)j * x.r + i] * ((q0 + q1) + (q2 + q3));
            }
        *out = s;
        return ST_OK;
    }

    int combine(int dst, const double* c, const int* src, int n) override {
        int m = 0;
        for (int t = 0; t < n; ++t) m += v_[src[t]].r;
        double* W;
        if (int st = scratch(0, m, &W)) return fail(st);
        std::vector<double> Q((size_t)nt_ * std::max(m, 1), 0.0);
        int off = 0;
        for (int t = 0; t < n; ++t) {
            const LrVec& x = v_[src[t]];
            if (x.r == 0) continue;
            if (cudaMemcpyAsync(W + (size_t)off * n_, x.P, sizeof(double) * n_ * x.r, cudaMemcpyDeviceToDevice,
                                c_.s) != cudaSuccess)
                return fail(ST_ECUDA);
            for (int j = 0; j < x.r; ++j)
                for (int l = 0; l < nt_; ++l) Q[(size_t)(off + j) * nt_ + l] = c[t] * x.Q[(size_t)j * nt_ + l];
            off += x.r;
        }
        return truncate_into(dst, W, m, Q);
    }

    int apply(int dst, int src) override {
        const LrVec& x = v_[src];
        const int r = x.r;
        double* W;
        if (int st = scratch(0, 2 * r, &W)) return fail(st);
        if (r > 0 && st_spmm_ma<double>(p_, x.P, n_, r, W, n_, W + (size_t)n_ * r, n_, c_.s) != ST_OK)
            return fail(ST_ECUDA);
        // [D_t Q, C_t Q]: (D_t q)_l = q_l - q_{l-1}, (C_t q)_l = dt/2 (q_l + q_{l-1})
        std::vector<double> Q((size_t)nt_ * std::max(2 * r, 1), 0.0);
        const double hdt = 0.5 * p_->dt;
        for (int j = 0; j < r; ++j)
            for (int l = 0; l < nt_; ++l) {
                const double q = x.Q[(size_t)j * nt_ + l], qp = l > 0 ? x.Q[(size_t)j * nt_ + l - 1] : 0.0;
                Q[(size_t)j * nt_ + l] = q - qp;
                Q[(size_t)(r + j) * nt_ + l] = hdt * (q + qp);
            }
        return truncate_into(dst, W, 2 * r, Q);
    }

    int precondition(int dst, int src) override {
        const LrVec& x = v_[src];
        if (x.r == 0) {
            v_[dst].r = 0;
            v_[dst].Q.clear();
            return ST_OK;
        }
        // RKSM on L(Z) = X with X's factors as (F1, F2), blocks of at most 16 columns, results summed
        std::vector<double> Qall;
        int m = 0;
        double* W = nullptr;
        std::vector<std::pair<int, int>> blocks;
        for (int j0 = 0; j0 < x.r; j0 += 16) blocks.push_back({j0, std::min(16, x.r - j0)});
        std::vector<std::vector<double>> Ys;
        std::vector<int> ks;
        std::vector<double*> Vs;
        for (auto [j0, cols] : blocks) {
            st_desc saved = p_->d;
            p_->d.maxit = piters_;
            p_->d.tol = 0.0;   // a fixed number of shifted solves
            st_solution sol{};
            st_stats ss{};
            double* F1 = x.P + (size_t)j0 * n_;
            const int rc = solve_impl(p_, F1, n_, &x.Q[(size_t)j0 * nt_], nt_, cols, &sol, &ss);
            p_->d = saved;
            if (rc != ST_OK && rc != ST_ENOTCONV && rc != ST_EBREAKDOWN) return fail(rc);
            pits_ += ss.iterations;
            const int k = sol.k;
            // keep V (the handle's basis is reused by the next block) and Y^T
            double* Vk;
            if (int st = scratch(1 + (int)Vs.size(), k, &Vk)) return fail(st);
            if (k > 0 && cudaMemcpyAsync(Vk, sol.V, sizeof(double) * n_ * k, cudaMemcpyDeviceToDevice, c_.s) !=
                             cudaSuccess)
                return fail(ST_ECUDA);
            std::vector<double> Y((size_t)std::max(k, 1) * nt_);
            if (k > 0)
                if (int st = read_dev(c_, sol.Y, k, k, nt_, Y.data(), k)) return fail(st);
            Vs.push_back(Vk);
            Ys.push_back(std::move(Y));
            ks.push_back(k);
            m += k;
        }
        if (int st = scratch(0, m, &W)) return fail(st);
        Qall.assign((size_t)nt_ * std::max(m, 1), 0.0);
        int off = 0;
        for (size_t b = 0; b < Vs.size(); ++b) {
            const int k = ks[b];
            if (k == 0) continue;
            if (cudaMemcpyAsync(W + (size_t)off * n_, Vs[b], sizeof(double) * n_ * k, cudaMemcpyDeviceToDevice,
                                c_.s) != cudaSuccess)
                return fail(ST_ECUDA);
            for (int j = 0; j < k; ++j)   // Q = Y^T
                for (int l = 0; l < nt_; ++l) Qall[(size_t)(off + j) * nt_ + l] = Ys[b][(size_t)l * k + j];
            off += k;
        }
        return truncate_into(dst, W, m, Qall);
    }

    int rank(int id) const override {
        auto it = v_.find(id);
        return it == v_.end() ? 0 : it->second.r;
    }

   private:
    int fail(int st) {
        if (st_ == ST_OK) st_ = st;
        return st;
    }

    int reserve(LrVec& x, int r) {
        if (r <= x.cap) return ST_OK;
        const int cap = std::max(r, 2 * x.cap);
        double* np = nullptr;
        ST_TRY(st_alloc(p_, (void**)&np, sizeof(double) * (size_t)n_ * cap));
        if (x.P) st_free_one(p_, x.P);   // stream-ordered: earlier work on the old buffer finishes first
        x.P = np;
        x.cap = cap;
        return ST_OK;
    }

    // device scratch buffer `id` of at least cols columns (contents not kept)
    int scratch(int id, int cols, double** out) {
        if ((int)scratch_.size() <= id) {
            scratch_.resize(id + 1, nullptr);
            scratch_cols_.resize(id + 1, 0);
        }
        if (scratch_cols_[id] < cols) {
            if (scratch_[id]) st_free_one(p_, scratch_[id]);
            scratch_[id] = nullptr;
            scratch_cols_[id] = 0;
            const int cap = std::max(cols, 16);
            ST_TRY(st_alloc(p_, (void**)&scratch_[id], sizeof(double) * (size_t)n_ * cap));
            scratch_cols_[id] = cap;
        }
        *out = scratch_[id];
        return ST_OK;
    }

    // W (device, n x m, overwritten) and Q (host, nt x m): X_dst = truncation of W Q^T.
    int truncate_into(int dst, double* W, int m, const std::vector<double>& Q) {
        LrVec& x = v_[dst];
        if (m == 0) {
            x.r = 0;
            x.Q.clear();
            return ST_OK;
        }
        if (m > nt_) {
            // more columns than time steps (sums of several full-rank-in-time vectors): the rank is at most
            // N_t, so form Z = W Q^T (N_h x N_t) by one dense product and truncate Z I^T instead; the column
            // QR then runs over N_t columns rather than m
            std::vector<double> QT((size_t)m * nt_);
            for (int j = 0; j < m; ++j)
                for (int l = 0; l < nt_; ++l) QT[(size_t)l * m + j] = Q[(size_t)j * nt_ + l];
            double *Z, *QTd;
            if (int st = scratch(kScratchZ, nt_, &Z)) return fail(st);
            if (int st = scratch(kScratchQT, (int)(((size_t)m * nt_ + n_ - 1) / n_), &QTd)) return fail(st);
            if (int st = write_dev(c_, QT.data(), m, m, nt_, QTd, m)) return fail(st);
            if (int st = st_lowrank_dense(n_, m, nt_, W, n_, QTd, m, Z, n_, c_.s)) return fail(st);
            std::vector<double> I((size_t)nt_ * nt_, 0.0);
            for (int l = 0; l < nt_; ++l) I[(size_t)l * nt_ + l] = 1.0;
            return truncate_into(dst, Z, nt_, I);
        }
        // column-wise QR of W: W = Q_W R (R m x m upper over the kept columns, zero rows elsewhere);
        // kept columns packed to the front, the rest zeroed
        std::vector<double> R((size_t)m * m, 0.0);
        int kept = 0;
        std::vector<double> h, nu2(1);
        for (int j = 0; j < m; ++j) {
            double* w = W + (size_t)kept * n_;
            if (kept != j && cudaMemcpyAsync(w, W + (size_t)j * n_, sizeof(double) * n_, cudaMemcpyDeviceToDevice,
                                             c_.s) != cudaSuccess)
                return fail(ST_ECUDA);
            if (int st = ts_tn_host(c_, 1, 1, w, n_, w, n_, nu2.data())) return fail(st);
            const double nu0 = std::sqrt(std::max(nu2[0], 0.0));
            double nu = nu0;
            std::vector<double> coef((size_t)std::max(kept, 1), 0.0);
            for (int pass = 0; pass < 4 && kept > 0 && nu > 0.0; ++pass) {
                h.assign(kept, 0.0);
                if (int st = ts_tn_host(c_, kept, 1, W, n_, w, n_, h.data())) return fail(st);
                if (int st = ts_nn_host(c_, kept, 1, -1.0, W, n_, h.data(), 1.0, w, n_)) return fail(st);
                for (int i = 0; i < kept; ++i) coef[i] += h[i];
                if (int st = ts_tn_host(c_, 1, 1, w, n_, w, n_, nu2.data())) return fail(st);
                const double nn = std::sqrt(std::max(nu2[0], 0.0));
                const bool settled = nn > 0.5 * nu;
                nu = nn;
                if (settled) break;
            }
            for (int i = 0; i < kept; ++i) R[(size_t)j * m + i] = coef[i];
            if (nu > 1e-13 * nu0 && nu > 0.0) {
                if (st_axpby64(n_, 1, 1.0 / nu, w, n_, 0.0, w, n_, c_.s) != ST_OK) return fail(ST_ECUDA);
                R[(size_t)j * m + kept] = nu;
                ++kept;
            }
        }
        if (kept < m && cudaMemsetAsync(W + (size_t)kept * n_, 0, sizeof(double) * n_ * (m - kept), c_.s) !=
                            cudaSuccess)
            return fail(ST_ECUDA);
        std::vector<double> Cp, Qn;
        int k = 0;
        lrgmres::truncate_core(m, R.data(), m, nt_, Q.data(), nt_, trunc_, dense::svd_small, dense::thin_qr, &Cp,
                               &Qn, &k);
        if (int st = reserve(x, k)) return fail(st);
        if (k > 0) {
            // P' = Q_W Cp (m x k)
            if (int st = ts_nn_host(c_, m, k, 1.0, W, n_, Cp.data(), 0.0, x.P, n_)) return fail(st);
        }
        x.r = k;
        x.Q = std::move(Qn);
        return ST_OK;
    }

    static constexpr int kScratchZ = 90, kScratchQT = 91;   // ids of the dense-product scratch buffers
    st_problem* p_;
    Ctx c_;
    int n_, nt_;
    double trunc_;
    int piters_;
    int pits_ = 0;
    int st_ = ST_OK;
    std::map<int, LrVec> v_;
    std::vector<double*> scratch_;
    std::vector<int> scratch_cols_;
};

}  // namespace

extern "C" int st_solve_lrfgmres(st_problem* p, const double* F1, int ldf1, const double* F2, int ldf2, int ncols,
                                 int maxit, int precond_iters, double trunc, st_solution* sol, st_stats* stats) {
    if (!p || !F1 || !F2 || ncols < 1 || ldf1 < p->n_h || ldf2 < p->n_t || maxit < 1 || precond_iters < 0 ||
        !(trunc >= 0.0))
        return ST_EINVAL;
    if (!p->tensor_heat && !(p->dim == 0 && p->d.op == ST_HEAT)) {
        st_note_msg("st_solve_lrfgmres: the RKSM preconditioner needs a heat problem (box grid or CSR matrices)");
        return ST_ENOTSUP;
    }
    const auto t0 = Clock::now();
    hostpar::ActiveSolve active;
    Ctx c{p, p->stream, p->n_h};
    const int n = p->n_h, nt = p->n_t;
    // the load's factors on the device and the host
    double* F1d = nullptr;
    ST_TRY(st_alloc(p, (void**)&F1d, sizeof(double) * (size_t)n * ncols));
    ST_TRY(st_stage_matrix(p, F1, ldf1, n, ncols, F1d));
    std::vector<double> F2h((size_t)nt * ncols);
    if (st_is_device_ptr(F2)) {
        ST_TRY(read_dev(c, F2, ldf2, nt, ncols, F2h.data(), nt));
    } else {
        for (int j = 0; j < ncols; ++j) std::memcpy(&F2h[(size_t)j * nt], F2 + (size_t)j * ldf2, sizeof(double) * nt);
    }
    st_stats S{};
    int rc = ST_OK;
    lrgmres::Result res;
    int k = 0;
    {
        DeviceBackend b(p, trunc, precond_iters);
        const int rhs = 0, x = 1;
        rc = b.set(rhs, F1d, n, F2h.data(), nt, ncols);
        lrgmres::Options o;
        o.tol = p->d.tol;
        o.maxit = maxit;
        if (rc == ST_OK) rc = lrgmres::run(b, rhs, x, o, &res);
        if (rc != ST_OK && b.status() != ST_OK) rc = b.status();
        if (rc == ST_OK) {
            // the solution U = P Q^T into the handle's output (V = P, Y = Q^T)
            LrVec& X = b.at(x);
            k = X.r;
            double* MV;
            if (k > 0) rc = ensure_basis(p, c, k, 0, &MV);
            if (rc == ST_OK && k > 0)
                if (cudaMemcpyAsync(p->V, X.P, sizeof(double) * (size_t)n * k, cudaMemcpyDeviceToDevice, c.s) !=
                    cudaSuccess)
                    rc = ST_ECUDA;
            if (rc == ST_OK && k > 0 && p->Y_cap < (size_t)k * nt) {
                if (p->Y) st_free_one(p, p->Y);
                p->Y = nullptr;
                p->Y_cap = 0;
                rc = st_alloc(p, (void**)&p->Y, sizeof(double) * (size_t)k * nt);
                if (rc == ST_OK) p->Y_cap = (size_t)k * nt;
            }
            if (rc == ST_OK && k > 0) {
                std::vector<double> Yh((size_t)k * nt);
                for (int j = 0; j < k; ++j)
                    for (int l = 0; l < nt; ++l) Yh[(size_t)l * k + j] = X.Q[(size_t)j * nt + l];
                rc = write_dev(c, Yh.data(), k, k, nt, p->Y, k);
            }
            p->k = k;
            S.inner_iterations = b.precond_iterations();
        }
        if (rc == ST_OK) {
            cudaError_t e = cudaStreamSynchronize(c.s);   // the backend's buffers are freed below
            if (e != cudaSuccess) rc = ST_ECUDA;
        }
    }
    st_free_one(p, F1d);
    if (rc != ST_OK) return rc;
    if (sol) {
        sol->n_h = n;
        sol->n_t = nt;
        sol->k = k;
        sol->V = p->V;
        sol->Y = p->Y;
        if (sol->U_dense) {
            if (sol->ldu < n) return ST_EINVAL;
            if (k > 0)
                ST_TRY(st_lowrank_dense(n, k, nt, p->V, n, p->Y, k, sol->U_dense, sol->ldu, c.s));
            else
                for (int l = 0; l < nt; ++l)
                    ST_CUDA_TRY(cudaMemsetAsync(sol->U_dense + (size_t)l * sol->ldu, 0, sizeof(double) * n, c.s));
            ST_CUDA_TRY(cudaStreamSynchronize(c.s));
        }
    }
    S.iterations = res.iterations;
    S.basis_cols = k;
    S.mu_mem = res.mu_mem;
    S.converged = res.converged ? 1 : 0;
    S.relres = res.history.empty() ? 0.0 : res.history.back();
    S.p = ncols;
    S.ms_total = std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
    if (stats) *stats = S;
    return res.converged ? ST_OK : ST_ENOTCONV;
}
