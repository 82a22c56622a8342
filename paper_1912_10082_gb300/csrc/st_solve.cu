// Rational Krylov Galerkin projection (RKSM) for M U D_t^T + A U C_t^T = F1 F2^T
// (paper Section 4, heat part), residuals, and the shifted-solve entry point.
//
// Device work: everything of size N_h (shifted solves, Gram-Schmidt, SpMM,
// projections).  Host work (Grace cores): the k x k projected problems, the
// adaptive shifts and the time recurrence of the projected equation.
#include <algorithm>
#include <array>
#include <cstdio>
#include <chrono>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "st_common.cuh"
#include "st_rksm.h"
#include "st_tune.h"

int st_slot(st_problem* p, int id, size_t bytes, void** out) {
    if (id < 0 || id >= 32) return ST_EINVAL;
    if (p->slot_bytes[id] < bytes) {
        // stream-ordered: work already issued on the stream finishes with the old buffer first
        if (p->slot_ptr[id]) st_free_one(p, p->slot_ptr[id]);
        p->slot_ptr[id] = nullptr;
        p->slot_bytes[id] = 0;
        ST_TRY(st_alloc(p, &p->slot_ptr[id], bytes));
        p->slot_bytes[id] = bytes;
    }
    *out = p->slot_ptr[id];
    return ST_OK;
}

namespace rksm {



// Records why the Krylov process broke down (text of st_last_error).
int breakdown(const char* why) {
    st_note_msg(why);
    return ST_EBREAKDOWN;
}


int read_dev(Ctx& c, const double* d, int ld, int rows, int cols, double* h, int ldh) {
    if (rows == 0 || cols == 0) return ST_OK;
    ST_CUDA_TRY(cudaMemcpy2DAsync(h, sizeof(double) * ldh, d, sizeof(double) * ld, sizeof(double) * rows, cols,
                                  cudaMemcpyDeviceToHost, c.s));
    ST_CUDA_TRY(cudaStreamSynchronize(c.s));
    return ST_OK;
}

int write_dev(Ctx& c, const double* h, int ldh, int rows, int cols, double* d, int ld) {
    if (rows == 0 || cols == 0) return ST_OK;
    ST_CUDA_TRY(cudaMemcpy2DAsync(d, sizeof(double) * ld, h, sizeof(double) * ldh, sizeof(double) * rows, cols,
                                  cudaMemcpyHostToDevice, c.s));
    return ST_OK;
}

// H (host, k x m) = V^T W over the n rows.
int ts_tn_host(Ctx& c, int k, int m, const double* V, int ldv, const double* W, int ldw, double* H) {
    if (k == 0 || m == 0) return ST_OK;
    double* dH;
    double* part;
    ST_TRY(st_slot(c.p, S_SMALL, sizeof(double) * (size_t)k * m, (void**)&dH));
    ST_TRY(st_slot(c.p, S_PART, sizeof(double) * st_tsgemm_partial_elems(c.n, k, m), (void**)&part));
    ST_TRY(st_tsgemm_tn(c.n, k, m, V, ldv, W, ldw, dH, k, part, c.s));
    return read_dev(c, dH, k, k, m, H, k);
}

// W = beta W + alpha V H with H given on the host (k x m).
int ts_nn_host(Ctx& c, int k, int m, double alpha, const double* V, int ldv, const double* H, double beta, double* W,
               int ldw) {
    if (m == 0) return ST_OK;
    double* dH;
    ST_TRY(st_slot(c.p, S_SMALL, sizeof(double) * (size_t)std::max(1, k) * m, (void**)&dH));
    ST_TRY(write_dev(c, H, k, k, m, dH, k));
    return st_tsgemm_nn(c.n, k, m, alpha, V, ldv, dH, k, beta, W, ldw, c.s);
}

// Orthonormalise the m columns of W (device) in place by CholQR2 with a
// rank-revealing fallback.  On return the first r columns hold Q and
// R (host, r x m, ld m) satisfies W_in = Q R up to directions whose norm is
// below drop * max(|W_in|, ref).  ref2 = squared norm of reference.
int block_qr(Ctx& c, double* W, int ldw, int m, double ref2, double drop, std::vector<double>& R, int* r_out) {
    *r_out = 0;
    R.assign((size_t)m * m, 0.0);
    if (m == 0) return ST_OK;
    std::vector<double> G((size_t)m * m), E((size_t)m * m), w(m);
    ST_TRY(ts_tn_host(c, m, m, W, ldw, W, ldw, G.data()));
    E = G;
    dense::sym_eig(m, E.data(), m, w.data());
    double lmax = std::max(w[m - 1], 0.0);
    double thr = drop * drop * std::max(lmax, ref2);
    int r = 0;
    for (int i = 0; i < m; ++i) r += w[i] > thr;
    if (r == 0) return ST_OK;
    double* dR;
    std::vector<double> L = G;
    // CholQR2 only for well-conditioned blocks (its first step loses cond(W)^2 u)
    bool full = (r == m) && w[0] > 1e-10 * lmax && dense::cholesky(m, L.data(), m);
    if (full) {
        // R1 = L^T; W <- W R1^{-1}; second pass
        std::vector<double> R1((size_t)m * m, 0.0);
        for (int j = 0; j < m; ++j)
            for (int i = 0; i <= j; ++i) R1[(size_t)j * m + i] = L[(size_t)i * m + j];
        ST_TRY(st_slot(c.p, S_SMALL, sizeof(double) * m * m, (void**)&dR));
        ST_TRY(write_dev(c, R1.data(), m, m, m, dR, m));
        ST_TRY(st_trsm_right_upper(c.n, m, dR, m, W, ldw, c.s));
        std::vector<double> G2((size_t)m * m);
        ST_TRY(ts_tn_host(c, m, m, W, ldw, W, ldw, G2.data()));
        if (!dense::cholesky(m, G2.data(), m)) return breakdown("block QR: second Gram matrix not positive definite");
        std::vector<double> R2((size_t)m * m, 0.0);
        for (int j = 0; j < m; ++j)
            for (int i = 0; i <= j; ++i) R2[(size_t)j * m + i] = G2[(size_t)i * m + j];
        ST_TRY(st_slot(c.p, S_SMALL, sizeof(double) * m * m, (void**)&dR));
        ST_TRY(write_dev(c, R2.data(), m, m, m, dR, m));
        ST_TRY(st_trsm_right_upper(c.n, m, dR, m, W, ldw, c.s));
        // R = R2 R1 (upper)
        for (int j = 0; j < m; ++j)
            for (int i = 0; i <= j; ++i) {
                double s = 0.0;
                for (int q = i; q <= j; ++q) s += R2[(size_t)q * m + i] * R1[(size_t)j * m + q];
                R[(size_t)j * m + i] = s;
            }
        *r_out = m;
        return ST_OK;
    }
    // ill-conditioned or rank-deficient: classical Gram-Schmidt twice, one column at a
    // time, each remainder's norm taken explicitly (not from a Gram matrix, whose small
    // eigenvalues carry only the absolute rounding of the large ones).  Kept directions
    // are packed into the first columns of W; R[:, j] holds column j's coordinates.
    double* copy;
    ST_TRY(st_slot(c.p, S_COPY, sizeof(double) * (size_t)c.n * m, (void**)&copy));
    ST_TRY(st_copy_cols64(c.n, m, W, ldw, copy, c.n, c.s));
    const double keep2 = drop * drop * std::max(lmax, ref2);
    int kept = 0;
    std::vector<double> h, h2;
    for (int j = 0; j < m; ++j) {
        double* wj = W + (size_t)kept * ldw;   // work column: the next free slot of W
        ST_TRY(st_copy_cols64(c.n, 1, copy + (size_t)j * c.n, c.n, wj, ldw, c.s));
        std::vector<double> coef(kept, 0.0);
        for (int pass = 0; pass < 2 && kept > 0; ++pass) {
            h.assign(kept, 0.0);
            ST_TRY(ts_tn_host(c, kept, 1, W, ldw, wj, ldw, h.data()));
            ST_TRY(ts_nn_host(c, kept, 1, -1.0, W, ldw, h.data(), 1.0, wj, ldw));
            for (int i = 0; i < kept; ++i) coef[i] += h[i];
        }
        h2.assign(1, 0.0);
        ST_TRY(ts_tn_host(c, 1, 1, wj, ldw, wj, ldw, h2.data()));
        for (int i = 0; i < kept; ++i) R[(size_t)j * m + i] = coef[i];
        if (h2[0] > keep2) {
            const double nrm = std::sqrt(h2[0]);
            ST_TRY(st_axpby64(c.n, 1, 1.0 / nrm, wj, ldw, 0.0, wj, ldw, c.s));
            R[(size_t)j * m + kept] = nrm;
            ++kept;
        }
    }
    *r_out = kept;
    return ST_OK;
}

// Shifted solve W = (A + s M)^{-1} M X (ncols columns), FP64 or FP32 + one FP64 refinement.
// MX, if given, holds M X already (used by the refinement residual).
int shifted_solve(Ctx& c, int prec, double shift, const double* X, int ldx, const double* MX, int ldmx, int ncols,
                  double* W, int ldw) {
    st_problem* p = c.p;
    size_t nm = (size_t)c.n * ncols;
    if (p->dim == 0) {
        // CSR problem: (A + s M) W = M X by the algebraic inner solver, to 1e-12 relative per column
        if (!MX) {
            double* mx;
            ST_TRY(st_slot(p, S_TMP, sizeof(double) * nm, (void**)&mx));
            ST_TRY(st_spmm_comb64(p, 1.0, 0.0, X, ldx, ncols, 0.0, mx, c.n, c.s));
            MX = mx;
            ldmx = c.n;
        }
        int its = 0;
        return pcg_solve(c, shift, 1.0, MX, ldmx, ncols, W, ldw, 1e-12, 50000, &its);
    }
    if (prec == ST_FP64) {
        double* tmp;
        ST_TRY(st_slot(p, S_TMP, sizeof(double) * nm, (void**)&tmp));
        return st_fd_apply64(p, FD_MASS_RESOLVENT, shift, 1.0, X, ldx, ncols, W, ldw, tmp, c.s);
    }
    float *x32, *w32, *t32;
    double* r64;
    ST_TRY(st_slot(p, S_X32, sizeof(float) * nm, (void**)&x32));
    ST_TRY(st_slot(p, S_W32, sizeof(float) * nm, (void**)&w32));
    ST_TRY(st_slot(p, S_T32, sizeof(float) * nm, (void**)&t32));
    ST_TRY(st_slot(p, S_TMP, sizeof(double) * nm, (void**)&r64));
    ST_TRY(st_convert_64_32(c.n, ncols, X, ldx, x32, c.n, c.s));
    ST_TRY(st_fd_apply32(p, FD_MASS_RESOLVENT, shift, 1.0, x32, c.n, ncols, w32, c.n, t32, c.s));
    ST_TRY(st_convert_32_64_add(c.n, ncols, w32, c.n, W, ldw, 0.0, c.s));
    // r = M X - (A + s M) W, in FP64
    ST_TRY(st_spmm_comb64(p, -shift, -1.0, W, ldw, ncols, 0.0, r64, c.n, c.s));
    if (MX) {
        ST_TRY(st_axpby64(c.n, ncols, 1.0, MX, ldmx, 1.0, r64, c.n, c.s));
    } else {
        ST_TRY(st_spmm_comb64(p, 1.0, 0.0, X, ldx, ncols, 1.0, r64, c.n, c.s));
    }
    // W += (A + s M)^{-1} r
    ST_TRY(st_convert_64_32(c.n, ncols, r64, c.n, x32, c.n, c.s));
    ST_TRY(st_fd_apply32(p, FD_RESOLVENT, shift, 1.0, x32, c.n, ncols, w32, c.n, t32, c.s));
    ST_TRY(st_convert_32_64_add(c.n, ncols, w32, c.n, W, ldw, 1.0, c.s));
    return ST_OK;
}

// M^{-1} X for the start block, FP64 or FP32 + refinement.
int mass_inverse(Ctx& c, int prec, const double* X, int ldx, int ncols, double* W, int ldw) {
    st_problem* p = c.p;
    size_t nm = (size_t)c.n * ncols;
    if (p->dim == 0) {
        int its = 0;
        return pcg_solve(c, 1.0, 0.0, X, ldx, ncols, W, ldw, 1e-13, 20000, &its);
    }
    if (prec == ST_FP64) {
        double* tmp;
        ST_TRY(st_slot(p, S_TMP, sizeof(double) * nm, (void**)&tmp));
        return st_fd_apply64(p, FD_MASS_INVERSE, 0.0, 1.0, X, ldx, ncols, W, ldw, tmp, c.s);
    }
    float *x32, *w32, *t32;
    double* r64;
    ST_TRY(st_slot(p, S_X32, sizeof(float) * nm, (void**)&x32));
    ST_TRY(st_slot(p, S_W32, sizeof(float) * nm, (void**)&w32));
    ST_TRY(st_slot(p, S_T32, sizeof(float) * nm, (void**)&t32));
    ST_TRY(st_slot(p, S_TMP, sizeof(double) * nm, (void**)&r64));
    ST_TRY(st_convert_64_32(c.n, ncols, X, ldx, x32, c.n, c.s));
    ST_TRY(st_fd_apply32(p, FD_MASS_INVERSE, 0.0, 1.0, x32, c.n, ncols, w32, c.n, t32, c.s));
    ST_TRY(st_convert_32_64_add(c.n, ncols, w32, c.n, W, ldw, 0.0, c.s));
    for (int it = 0; it < 2; ++it) {
        ST_TRY(st_spmm_comb64(p, -1.0, 0.0, W, ldw, ncols, 0.0, r64, c.n, c.s));
        ST_TRY(st_axpby64(c.n, ncols, 1.0, X, ldx, 1.0, r64, c.n, c.s));
        ST_TRY(st_convert_64_32(c.n, ncols, r64, c.n, x32, c.n, c.s));
        ST_TRY(st_fd_apply32(p, FD_MASS_INVERSE, 0.0, 1.0, x32, c.n, ncols, w32, c.n, t32, c.s));
        ST_TRY(st_convert_32_64_add(c.n, ncols, w32, c.n, W, ldw, 1.0, c.s));
    }
    return ST_OK;
}

// log of prod_j |s - s_j| / prod_i |s + theta_i| (products renormalised to avoid overflow).
double shift_objective(double s, double b, const std::vector<double>& used, const std::vector<double>& ritz) {
    // numerator and denominator as separate products (multiplications only),
    // renormalised every 16 factors to stay in range
    const double ib = 1.0 / b;
    auto logprod = [&](const std::vector<double>& v, double sign) {
        double prod = 1.0;
        long long ex = 0;
        int cnt = 0;
        for (double t : v) {
            prod *= std::fabs(s + sign * t) * ib;
            if (++cnt == 16) {
                int e;
                prod = std::frexp(prod, &e);
                ex += e;
                cnt = 0;
            }
        }
        return prod > 0.0 ? std::log(prod) + (double)ex * std::log(2.0) : -1e300;
    };
    const double num = logprod(used, -1.0);
    if (num <= -1e299) return -1e300;
    const double den = logprod(ritz, 1.0);
    if (den <= -1e299) return -1e300;
    return num - den;
}

// Next shift by the adaptive rule: maximise prod_j |s - s_j| / prod_i |s + theta_i|
// over [a, b] on a log scale: a coarse grid of `grid` points, then a finer one
// over the two coarse cells around the best point.
double next_shift(double a, double b, const std::vector<double>& used, const std::vector<double>& ritz, int grid) {
    double la = std::log(a), lb = std::log(b);
    double step = (lb - la) / (grid - 1);
    int gbest = 0;
    double bestv = -1e300;
    for (int g = 0; g < grid; ++g) {
        double v = shift_objective(std::exp(la + step * g), b, used, ritz);
        if (v > bestv) {
            bestv = v;
            gbest = g;
        }
    }
    double best = std::exp(la + step * gbest);
    double lo = la + step * std::max(0, gbest - 1), hi = la + step * std::min(grid - 1, gbest + 1);
    const int fine = 48;
    for (int g = 0; g <= fine; ++g) {
        double sv = std::exp(lo + (hi - lo) * g / fine);
        double v = shift_objective(sv, b, used, ritz);
        if (v > bestv) {
            bestv = v;
            best = sv;
        }
    }
    return best;
}

// Ritz values of the pencil (Am, Mm): eigenvalues of L^{-1} Am L^{-T}, Mm = L L^T.
bool ritz_values(int k, const double* Am, const double* Mm, int ld, std::vector<double>& out) {
    std::vector<double> L((size_t)k * k), C((size_t)k * k);
    for (int j = 0; j < k; ++j)
        for (int i = 0; i < k; ++i) {
            L[(size_t)j * k + i] = Mm[(size_t)j * ld + i];
            C[(size_t)j * k + i] = Am[(size_t)j * ld + i];
        }
    if (!dense::cholesky(k, L.data(), k)) return false;
    // X = L^{-1} C (column by column), then C = L^{-1} X^T
    for (int pass = 0; pass < 2; ++pass) {
        dense::lower_solve(k, L.data(), k, C.data(), k, k);
        for (int j = 0; j < k; ++j)
            for (int i = j + 1; i < k; ++i) std::swap(C[(size_t)j * k + i], C[(size_t)i * k + j]);
    }
    for (int j = 0; j < k; ++j)
        for (int i = j + 1; i < k; ++i) {
            double v = 0.5 * (C[(size_t)j * k + i] + C[(size_t)i * k + j]);
            C[(size_t)j * k + i] = v;
            C[(size_t)i * k + j] = v;
        }
    out.resize(k);
    dense::sym_eigvals(k, C.data(), k, out.data());
    return true;
}

// Projected equation Mm Y D_t^T + Am Y C_t^T = Gm F2c^T (k x n_t), by the time
// recurrence of the lower-bidiagonal time pencil:
// (Mm + dt/2 Am) y_l = Gm F2c[l, :]^T + (Mm - dt/2 Am) y_{l-1}.
// With P = Mm + dt/2 Am factored once, S = P^{-1}(Mm - dt/2 Am) and
// G = P^{-1} Gm are formed first, so each step costs one k x k product.
bool projected_solve(int k, int n_t, double dt, const double* Mm, const double* Am, int ld, const double* Gm,
                     int ldg, int r, const double* F2c, std::vector<double>& Y, bool sym) {
    std::vector<double> P((size_t)k * k), S((size_t)k * k), G((size_t)k * r);
    for (int j = 0; j < k; ++j)
        for (int i = 0; i < k; ++i) {
            double m = Mm[(size_t)j * ld + i], a = Am[(size_t)j * ld + i];
            P[(size_t)j * k + i] = m + 0.5 * dt * a;
            S[(size_t)j * k + i] = m - 0.5 * dt * a;
        }
    for (int q = 0; q < r; ++q)
        for (int i = 0; i < k; ++i) G[(size_t)q * k + i] = Gm[(size_t)q * ldg + i];
    if (sym) {
        if (!dense::cholesky(k, P.data(), k)) return false;
        dense::chol_solve(k, P.data(), k, S.data(), k, k);
        dense::chol_solve(k, P.data(), k, G.data(), k, r);
    } else {
        std::vector<int> piv(k);
        if (!dense::lu(k, P.data(), k, piv.data())) return false;
        dense::lu_solve(k, P.data(), k, piv.data(), S.data(), k, k);
        dense::lu_solve(k, P.data(), k, piv.data(), G.data(), k, r);
    }
    Y.assign((size_t)k * n_t, 0.0);
    // the rows of each step split over a thread team, a barrier between steps
    const int T = hostpar::threads_for(2.0 * k * k * n_t);
    hostpar::run(T, [&](int t, hostpar::Barrier& bar) {
        const int i0 = (int)((long long)k * t / T), i1 = (int)((long long)k * (t + 1) / T);
        for (int l = 0; l < n_t; ++l) {
            double* y = &Y[(size_t)l * k];
            for (int q = 0; q < r; ++q) {
                double f = F2c[(size_t)q * n_t + l];
                const double* gq = &G[(size_t)q * k];
                for (int i = i0; i < i1; ++i) y[i] += gq[i] * f;
            }
            if (l > 0) {
                const double* yp = y - k;
                for (int j = 0; j < k; ++j) {
                    double tj = yp[j];
                    const double* sc = &S[(size_t)j * k];
                    for (int i = i0; i < i1; ++i) y[i] += sc[i] * tj;
                }
            }
            bar.wait();
        }
    });
    return true;
}

int ensure_basis(st_problem* p, Ctx& c, int need_cols, int keep_cols, double** MV) {
    if ((size_t)need_cols <= p->V_cap_cols && p->slot_bytes[S_MV] >= sizeof(double) * (size_t)c.n * need_cols) {
        *MV = (double*)p->slot_ptr[S_MV];
        return ST_OK;
    }
    // doubling while the basis is small; beyond 16M entries a column block, grow by half (the old and
    // new blocks coexist during the copy, so doubling a large basis triples its footprint)
    const size_t grown = (size_t)c.n * p->V_cap_cols <= ((size_t)1 << 24) ? 2 * p->V_cap_cols
                                                                             : p->V_cap_cols + p->V_cap_cols / 2;
    size_t cap = std::max<size_t>({(size_t)need_cols, grown, 32});
    cap = std::min<size_t>(cap, (size_t)p->d.max_basis + 16);
    if (cap < (size_t)need_cols) cap = need_cols;
    double *nv, *nmv;
    float2* ndf = nullptr;
    ST_TRY(st_alloc(p, (void**)&nv, sizeof(double) * (size_t)c.n * cap));
    ST_TRY(st_alloc(p, (void**)&nmv, sizeof(double) * (size_t)c.n * cap));
    if (p->d.precision == ST_MIXED) ST_TRY(st_alloc(p, (void**)&ndf, sizeof(float2) * (size_t)c.n * cap));
    if (keep_cols > 0) {
        ST_CUDA_TRY(cudaMemcpyAsync(nv, p->V, sizeof(double) * (size_t)c.n * keep_cols, cudaMemcpyDeviceToDevice, c.s));
        ST_CUDA_TRY(cudaMemcpyAsync(nmv, p->slot_ptr[S_MV], sizeof(double) * (size_t)c.n * keep_cols,
                                    cudaMemcpyDeviceToDevice, c.s));
        if (ndf && p->Vdf)
            ST_CUDA_TRY(cudaMemcpyAsync(ndf, p->Vdf, sizeof(float2) * (size_t)c.n * keep_cols,
                                        cudaMemcpyDeviceToDevice, c.s));
    }
    // stream-ordered frees: they take effect after the copies above
    if (p->V) st_free_one(p, p->V);
    if (p->Vdf) st_free_one(p, p->Vdf);
    if (p->slot_ptr[S_MV]) st_free_one(p, p->slot_ptr[S_MV]);
    p->Vdf = ndf;
    p->V = nv;
    p->V_cap_cols = cap;
    p->slot_ptr[S_MV] = nmv;
    p->slot_bytes[S_MV] = sizeof(double) * (size_t)c.n * cap;
    *MV = nmv;
    return ST_OK;
}


// ---- staging of the small results of one synchronisation point ----
// The device buffer sm_dev holds a download region [0, cap) that collects the
// small products the host needs after the next synchronisation, and an upload
// region [cap, 2 cap) for small host matrices.  The host mirror is pinned, so
// every synchronisation point costs one device-to-host copy.
int stage_reserve(st_problem* p, size_t need) {
    if (p->sm_cap >= need) return ST_OK;
    size_t cap = std::max<size_t>({need, 2 * p->sm_cap, (size_t)8192});
    if (p->sm_dev || p->sm_host) ST_CUDA_TRY(cudaStreamSynchronize(p->stream));
    if (p->sm_dev) st_free_one(p, p->sm_dev);   // stream-ordered
    st_pinned_put(p->sm_host, p->sm_host_bytes);   // the stream is idle: no copy uses it
    p->sm_dev = nullptr;
    p->sm_host = nullptr;
    p->sm_cap = 0;
    p->sm_host_bytes = 0;
    ST_TRY(st_alloc(p, (void**)&p->sm_dev, sizeof(double) * 2 * cap));
    p->sm_host = (double*)st_pinned_get(sizeof(double) * 2 * cap, &p->sm_host_bytes);
    if (!p->sm_host) {
        st_note_msg("pinned host staging: allocation failed");
        p->sm_host_bytes = 0;
        return ST_ENOMEM;
    }
    p->sm_cap = cap;
    return ST_OK;
}


struct Stage {
    Ctx& c;
    size_t down = 0, up = 0;
    bool overflow = false;
    explicit Stage(Ctx& cc) : c(cc) {}
    // device address of the next m doubles of the download region.  Every
    // caller reserves its phase's total first; if that sizing were ever short,
    // the request is redirected to the start of the region (in bounds) and
    // the next fetch reports the error.
    double* out(size_t m) {
        if (down + pad32(m) > c.p->sm_cap) {
            overflow = true;
            return c.p->sm_dev;
        }
        double* d = c.p->sm_dev + down;
        down += pad32(m);
        return d;
    }
    bool fits() const { return !overflow && down <= c.p->sm_cap && up <= c.p->sm_cap; }
    const double* host_of(const double* d) const { return c.p->sm_host + (d - c.p->sm_dev); }
    // copies m host doubles to the device through the pinned upload region
    int in(const double* h, size_t m, double** d) {
        size_t off = c.p->sm_cap + up;
        if (up + pad32(m) > c.p->sm_cap) {
            st_note_msg("internal error: solver upload area sized too small");
            return ST_EINVAL;
        }
        up += pad32(m);
        std::memcpy(c.p->sm_host + off, h, sizeof(double) * m);
        ST_CUDA_TRY(cudaMemcpyAsync(c.p->sm_dev + off, c.p->sm_host + off, sizeof(double) * m,
                                    cudaMemcpyHostToDevice, c.s));
        *d = c.p->sm_dev + off;
        return ST_OK;
    }
    // one copy of the download region, then wait for the stream
    int fetch() {
        if (!fits()) {
            st_note_msg("internal error: solver staging area sized too small");
            return ST_EINVAL;
        }
        if (down) ST_CUDA_TRY(cudaMemcpyAsync(c.p->sm_host, c.p->sm_dev, sizeof(double) * down,
                                              cudaMemcpyDeviceToHost, c.s));
        ST_CUDA_TRY(cudaStreamSynchronize(c.s));
        down = 0;
        up = 0;
        return ST_OK;
    }
};

// H (device, k x m, ld ldh) = V^T W over the n rows.
int ts_tn_dev(Ctx& c, int k, int m, const double* V, int ldv, const double* W, int ldw, double* H, int ldh) {
    if (k == 0 || m == 0) return ST_OK;
    double* part;
    ST_TRY(st_slot(c.p, S_PART, sizeof(double) * st_tsgemm_partial_elems(c.n, k, m), (void**)&part));
    return st_tsgemm_tn(c.n, k, m, V, ldv, W, ldw, H, ldh, part, c.s);
}

// H (device) = V^T W and W -= V H against the first k basis columns: FP64, or
// double-float on the FP32 pipes when the solve is in mixed precision.
int basis_tn(Ctx& c, bool df, int k, int m, const double* W, int ldw, double* H, int ldh) {
    if (!df) return ts_tn_dev(c, k, m, c.p->V, c.n, W, ldw, H, ldh);
    if (k == 0 || m == 0) return ST_OK;
    double* part;
    float2* W2;
    ST_TRY(st_slot(c.p, S_PART, sizeof(double) * st_tsgemm_partial_elems(c.n, k, m), (void**)&part));
    ST_TRY(st_slot(c.p, S_WDF, sizeof(float2) * (size_t)c.n * m, (void**)&W2));
    ST_TRY(st_to_df(c.n, m, W, ldw, W2, c.n, c.s));
    return st_tsgemm_tn_df(c.n, k, m, c.p->Vdf, c.n, W2, c.n, H, ldh, part, c.s);
}

int basis_nn_sub(Ctx& c, bool df, int k, int m, const double* H, int ldh, double* W, int ldw) {
    if (!df) return st_tsgemm_nn(c.n, k, m, -1.0, c.p->V, c.n, H, ldh, 1.0, W, ldw, c.s);
    return st_tsgemm_nn_df(c.n, k, m, -1.0, c.p->Vdf, c.n, H, ldh, 1.0, W, ldw, c.s);
}

// Rank of a block from its Gram matrix G = W^T W (host, m x m) and, when it
// has full rank and a Cholesky factor, the first CholQR factor R1 = L^T.
// The rank counts the eigenvalues above drop^2 max(lambda_max, ref2), the
// rule of block_qr, which handles every block that is not of full rank.

void qr_plan(const double* G, int m, double ref2, double drop, QrPlan& q) {
    std::vector<double> E(G, G + (size_t)m * m), w(m);
    dense::sym_eigvals(m, E.data(), m, w.data());
    double lmax = std::max(w[m - 1], 0.0);
    double thr = drop * drop * std::max(lmax, ref2);
    q.rank = 0;
    double wkept = 0.0;
    for (int i = 0; i < m; ++i)
        if (w[i] > thr) {
            wkept = q.rank == 0 ? w[i] : std::min(wkept, w[i]);
            ++q.rank;
        }
    q.severe = q.rank > 0 && wkept < 1e-12 * std::max(lmax, ref2);
    // CholQR2 loses orthogonality like cond(W)^2 u in its first step: keep it to
    // blocks with cond(W) < ~1e5 (Gram eigenvalue ratio 1e-10, also the accuracy of
    // a double-float Gram matrix); the rest go to block_qr
    q.fast = false;
    if (q.rank == m && w[0] > 1e-10 * lmax) {
        std::vector<double> L(G, G + (size_t)m * m);
        if (dense::cholesky(m, L.data(), m)) {
            q.R1.assign((size_t)m * m, 0.0);
            for (int j = 0; j < m; ++j)
                for (int i = 0; i <= j; ++i) q.R1[(size_t)j * m + i] = L[(size_t)i * m + j];
            q.fast = true;
        }
    }
}

// Device part of CholQR2 for a full-rank block: W <- W R1^{-1}, then the
// second Gram matrix, its Cholesky factor R2 by one warp, W <- W R2^{-1}.
// R2 and the pivot flag land in the download region.
int qr_fast_launch(Ctx& c, Stage& sg, double* W, int ldw, int m, const std::vector<double>& R1, double** dR2,
                   double** dflag) {
    double* dR1;
    ST_TRY(sg.in(R1.data(), (size_t)m * m, &dR1));
    ST_TRY(st_trsm_right_upper(c.n, m, dR1, m, W, ldw, c.s));
    double* dG2 = sg.out((size_t)m * m);
    ST_TRY(ts_tn_dev(c, m, m, W, ldw, W, ldw, dG2, m));
    *dR2 = sg.out((size_t)m * m);
    *dflag = sg.out(1);
    ST_TRY(st_chol_small(m, dG2, m, *dR2, m, *dflag, c.s));
    ST_TRY(st_trsm_right_upper(c.n, m, *dR2, m, W, ldw, c.s));
    return ST_OK;
}

// R = R2 R1 for upper triangular m x m factors (ld m).
std::vector<double> upper_product(int m, const double* R2, const double* R1) {
    std::vector<double> R((size_t)m * m, 0.0);
    for (int j = 0; j < m; ++j)
        for (int i = 0; i <= j; ++i) {
            double s = 0.0;
            for (int q = i; q <= j; ++q) s += R2[(size_t)q * m + i] * R1[(size_t)j * m + q];
            R[(size_t)j * m + i] = s;
        }
    return R;
}

// Gram matrix Gb = b^T b of the residual direction b = w_hat - M V Mm^{-1} V^T w_hat,
// w_hat = -(s M q + A q) R_q (the rational Arnoldi residual), evaluated on the
// device (one extra synchronisation, taken only at residual checks).
int residual_gram_explicit(Ctx& c, int k, int pn, int pl, double s, const double* MAq, const double* MV,
                           const std::vector<double>& X1, const HostSym& Mm, const std::vector<double>& Rq,
                           std::vector<double>& Gb) {
    st_problem* p = c.p;
    const int n = c.n;
    double* Wh;
    double* Wh2;
    ST_TRY(st_slot(p, S_WH, sizeof(double) * (size_t)n * pl, (void**)&Wh));
    ST_TRY(st_slot(p, S_WH2, sizeof(double) * (size_t)n * pl, (void**)&Wh2));
    std::vector<double> negR((size_t)pn * pl);
    for (int j = 0; j < pl; ++j)
        for (int i = 0; i < pn; ++i) negR[(size_t)j * pn + i] = -Rq[(size_t)j * pl + i];
    ST_TRY(st_copy_cols64(n, pn, MAq + (size_t)n * pn, n, Wh, n, c.s));
    ST_TRY(st_axpby64(n, pn, s, MAq, n, 1.0, Wh, n, c.s));   // Wh = s Mq + Aq
    ST_TRY(ts_nn_host(c, pn, pl, 1.0, Wh, n, negR.data(), 0.0, Wh2, n));
    std::vector<double> Vw((size_t)k * pl, 0.0);
    for (int j = 0; j < pl; ++j)
        for (int q = 0; q < pn; ++q) {
            double rq = -Rq[(size_t)j * pl + q];
            for (int i = 0; i < k; ++i)
                Vw[(size_t)j * k + i] += (s * X1[(size_t)q * k + i] + X1[(size_t)(pn + q) * k + i]) * rq;
        }
    std::vector<double> L((size_t)k * k);
    for (int j = 0; j < k; ++j)
        for (int i = 0; i < k; ++i) L[(size_t)j * k + i] = Mm.a[(size_t)j * Mm.ld + i];
    if (!dense::cholesky(k, L.data(), k)) return breakdown("residual: projected mass matrix not positive definite");
    dense::chol_solve(k, L.data(), k, Vw.data(), k, pl);
    ST_TRY(ts_nn_host(c, k, pl, -1.0, MV, n, Vw.data(), 1.0, Wh2, n));
    Gb.assign((size_t)pl * pl, 0.0);
    return ts_tn_host(c, pl, pl, Wh2, n, Wh2, n, Gb.data());
}

// Iterations until the next residual check.  The projected solve of a check
// costs about k^2 n_t flops on the host.  Once two checks exist, the observed
// geometric rate predicts how many iterations remain to reach tol; the next
// check comes after about half of them, so the solve overshoots by little
// while checks stay rare.  Before that, or when the residual stagnates, a
// cost rule spaces the checks.
int check_gap(const std::vector<int>& hist_it, const std::vector<double>& hist_res, int it, double res, double tol,
              double cost) {
    int gap_cost = (int)std::max(1.0, std::min(16.0, cost / 4e6));
    if (hist_it.empty() || !(res > 0.0)) return gap_cost;
    double prev = hist_res.back();
    int dit = it - hist_it.back();
    if (dit <= 0 || !(prev > res)) return gap_cost;
    double rate = std::pow(res / prev, 1.0 / dit);   // per iteration, < 1
    double need = std::log(tol / res) / std::log(rate);
    int gap = (int)std::floor(0.5 * need);
    return std::max(1, std::min(gap, 24));
}

// Shifted solve (A + s M) W = M X for a nonsymmetric A (convection-diffusion):
// flexible GMRES, right-preconditioned by the x-line solve of
// eps K + beta_x Gx (x) M_rest + s M (y, z in sine modes, Thomas sweeps along x;
// exact in 1D) when beta_x is the largest convection component, else by the
// fast-diagonalisation solve of eps K + s M.  The preconditioned directions T_j
// are kept, so W = T y has exactly the GMRES residual whatever the
// preconditioner's precision.  The columns run as independent GMRES processes
// advanced together (each kernel covers the whole block, vectors interleaved):
// classical Gram-Schmidt twice, the new vector normalised on the device from
// the second pass's Gram products, so a step needs no synchronisation.  Every
// CHK steps the host fetches the new Hessenberg columns, applies the Givens
// rotations of each column and stops the cycle once every column has reached
// its target (a column that converged inside a CHK window uses only its own
// steps).  Restarts after J steps from the true residual, in FP64.
//
// TB = double: the Krylov vectors in FP64, each cycle aims at
// ||b - (A + sM) w|| <= rtol ||b||.  TB = float (mixed precision on large
// grids): iterative refinement.  The Arnoldi process, the operator product
// and the preconditioner run in FP32 on the FP64 true residual of the cycle
// (half the bytes, and FP32 instead of 1/64-rate FP64 arithmetic); a cycle
// aims at a 1e-5 reduction, its correction is added to w in FP64 and the next
// cycle starts from the new FP64 residual, until rtol ||b|| is met.
template <typename TB>
int fgmres_impl(Ctx& c, int prec, double shift, const double* X, int ldx, const double* MX, int ldmx, int ncols,
                double* W, int ldw, double rtol, int* iters_out) {
    constexpr bool IR = std::is_same<TB, float>::value;
    st_problem* p = c.p;
    const int n = c.n;
    constexpr int J = 40, CYCLES = 12, CHK = 4, MAXG = 16;
    constexpr double TAU = 1e-5;   // per-cycle reduction an FP32 inner solve aims at
    // columns per group: all of them (at most 16) unless the Krylov blocks would exceed 4 GB
    const double per_col = (double)sizeof(TB) * n * (2.0 * J + 4.0);
    const int mg = std::max(1, std::min({ncols, MAXG, (int)std::max(1.0, 4e9 / per_col)}));
    const long long ldhd = (long long)J * (J + 1);
    TB *Z, *T;
    double *B, *tmp, *Hc, *Hd, *part;
    ST_TRY(st_slot(p, S_GZ, sizeof(TB) * (size_t)n * (J + 1) * mg, (void**)&Z));
    ST_TRY(st_slot(p, S_GT, sizeof(TB) * (size_t)n * J * mg, (void**)&T));
    ST_TRY(st_slot(p, S_WH, sizeof(double) * (size_t)n * mg, (void**)&B));
    ST_TRY(st_slot(p, S_TMP, sizeof(double) * (size_t)n * mg, (void**)&tmp));   // IR: the FP64 residual
    ST_TRY(st_slot(p, S_GH, sizeof(double) * (size_t)2 * (J + 2) * mg, (void**)&Hc));
    ST_TRY(st_slot(p, S_GHD, sizeof(double) * (size_t)ldhd * mg, (void**)&Hd));
    ST_TRY(st_slot(p, S_GPART, sizeof(double) * st_gm_partial_elems(n, J + 2, mg), (void**)&part));
    double* H1 = Hc;                          // first pass coefficients, ld J + 2
    double* H2 = Hc + (size_t)(J + 2) * mg;   // second pass (and the squared norm at i = j + 1)
    double* R = IR ? tmp : nullptr;           // IR: FP64 residual of the cycle
    float *x32 = nullptr, *w32 = nullptr, *t32 = nullptr;
    if (prec == ST_MIXED) {
        ST_TRY(st_slot(p, S_X32, sizeof(float) * (size_t)n * mg, (void**)&x32));
        ST_TRY(st_slot(p, S_W32, sizeof(float) * (size_t)n * mg, (void**)&w32));
        ST_TRY(st_slot(p, S_T32, sizeof(float) * (size_t)n * mg, (void**)&t32));
    }
    // preconditioner: the x-line solve (x convection kept) when beta_x is the largest
    // component, else the fast-diagonalisation solve of eps K + s M
    const bool line = st_line_usable(p);
    if (line) ST_TRY(st_line_factor(p, shift, c.s));
    auto precond = [&](const TB* z, TB* t, int m) -> int {
        if constexpr (IR) {
            if (line) return st_line_apply32(p, 1.0, z, n, m, t, n, t32, c.s);
            return st_fd_apply32(p, FD_RESOLVENT, shift, 1.0, z, n, m, t, n, t32, c.s);
        } else {
            if (prec != ST_MIXED) {
                if (line) return st_line_apply64(p, 1.0, z, n, m, t, n, tmp, c.s);
                return st_fd_apply64(p, FD_RESOLVENT, shift, 1.0, z, n, m, t, n, tmp, c.s);
            }
            ST_TRY(st_convert_64_32(n, m, z, n, x32, n, c.s));
            if (line)
                ST_TRY(st_line_apply32(p, 1.0, x32, n, m, w32, n, t32, c.s));
            else
                ST_TRY(st_fd_apply32(p, FD_RESOLVENT, shift, 1.0, x32, n, m, w32, n, t32, c.s));
            return st_convert_32_64_add(n, m, w32, n, t, n, 0.0, c.s);
        }
    };
    auto op = [&](const TB* t, TB* u, int m) -> int {
        if constexpr (IR)
            return st_spmm_comb32(p, shift, 1.0, t, n, m, u, n, c.s);
        else
            return st_spmm_comb64(p, shift, 1.0, t, n, m, 0.0, u, n, c.s);
    };
    ST_TRY(stage_reserve(p, pad32((size_t)mg * ldhd) + pad32((size_t)(J + 2) * mg) + pad32((size_t)J * mg) +
                                2 * pad32(mg)));
    Stage sg(c);
    int total = 0;
    struct ColState {
        std::vector<double> H, cs, sn, g;
        double bnorm = -1.0, beta = 0.0;
        bool active = false, conv = false;
        int used = 0;   // Arnoldi steps of this cycle that enter the solution
    };
    std::vector<ColState> cols(mg);
    for (auto& cl : cols) {
        cl.H.assign((size_t)(J + 1) * J, 0.0);
        cl.cs.assign(J, 0.0);
        cl.sn.assign(J, 0.0);
        cl.g.assign(J + 1, 0.0);
    }
    std::vector<double> f(mg), y(J), ys((size_t)J * mg);
    for (int g0 = 0; g0 < ncols; g0 += mg) {
        const int m = std::min(mg, ncols - g0);
        double* Wg = W + (size_t)g0 * ldw;
        if (MX) {
            ST_TRY(st_copy_cols64(n, m, MX + (size_t)g0 * ldmx, ldmx, B, n, c.s));
        } else {
            ST_TRY(st_spmm_ma<double>(p, X + (size_t)g0 * ldx, ldx, m, B, n, (double*)nullptr, n, c.s));
        }
        for (int k = 0; k < m; ++k) ST_CUDA_TRY(cudaMemsetAsync(Wg + (size_t)k * ldw, 0, sizeof(double) * n, c.s));
        if constexpr (IR)
            ST_TRY(st_copy_cols64(n, m, B, n, R, n, c.s));   // R = B
        else
            ST_TRY(st_copy_cols64(n, m, B, n, Z, n, c.s));   // R = B in vector 0
        for (int k = 0; k < m; ++k) cols[k].bnorm = -1.0;
        for (int cyc = 0; cyc < CYCLES; ++cyc) {
            // residual norms of the block (FP64)
            if constexpr (IR)
                ST_TRY(st_gm_dots<double>(n, 1, m, R, part, H2, J + 2, c.s));
            else
                ST_TRY(st_gm_dots<double>(n, 1, m, Z, part, H2, J + 2, c.s));
            double* dn = sg.out(m);
            ST_CUDA_TRY(cudaMemcpy2DAsync(dn, sizeof(double), H2, sizeof(double) * (J + 2), sizeof(double), m,
                                          cudaMemcpyDeviceToDevice, c.s));
            ST_TRY(sg.fetch());
            bool any = false;
            for (int k = 0; k < m; ++k) {
                ColState& cl = cols[k];
                cl.beta = std::sqrt(std::max(sg.host_of(dn)[k], 0.0));
                if (cl.bnorm < 0) cl.bnorm = cl.beta;
                cl.active = cl.beta > rtol * cl.bnorm && cl.beta > 0.0;
                cl.conv = !cl.active;
                cl.used = 0;
                std::fill(cl.g.begin(), cl.g.end(), 0.0);
                cl.g[0] = cl.beta;
                f[k] = cl.active ? 1.0 / cl.beta : 0.0;
                any = any || cl.active;
            }
            if (!any) break;
            double* df;
            ST_TRY(sg.in(f.data(), m, &df));
            if constexpr (IR)
                ST_TRY(st_scale_cols_to32(n, m, R, n, df, Z, n, c.s));
            else
                ST_TRY(st_scale_cols_dev(n, m, Z, n, df, c.s));
            int j = 0, checked = 0;
            bool all_conv = false;
            for (; j < J && !all_conv; ++j) {
                TB* Zj = Z + (size_t)j * m * n;
                TB* Tj = T + (size_t)j * m * n;
                TB* U = Z + (size_t)(j + 1) * m * n;
                ST_TRY(precond(Zj, Tj, m));
                ST_TRY(op(Tj, U, m));
                ST_TRY(st_gm_dots<TB>(n, j + 2, m, Z, part, H1, J + 2, c.s));
                // first pass's update and second pass's dots in one sweep of the basis
                ST_TRY(st_gm_update_dot<TB>(n, j + 1, m, Z, H1, J + 2, part, H2, J + 2, c.s));
                ST_TRY(st_gm_update<TB>(n, j + 1, m, Z, H2, J + 2, H1, J + 2, Hd, ldhd, j, J, c.s));
                if ((j + 1) % CHK != 0 && j + 1 < J) continue;
                // Hessenberg columns checked..j of every column of the block
                const int nc = j + 1 - checked;
                double* dh = sg.out((size_t)m * ldhd);
                for (int k = 0; k < m; ++k)
                    ST_CUDA_TRY(cudaMemcpyAsync(dh + (size_t)k * ldhd + (size_t)checked * (J + 1),
                                                Hd + (size_t)k * ldhd + (size_t)checked * (J + 1),
                                                sizeof(double) * (size_t)nc * (J + 1), cudaMemcpyDeviceToDevice, c.s));
                ST_TRY(sg.fetch());
                all_conv = true;
                for (int k = 0; k < m; ++k) {
                    ColState& cl = cols[k];
                    if (!cl.active || cl.conv) continue;
                    const double target = IR ? std::max(rtol * cl.bnorm, TAU * cl.beta) : rtol * cl.bnorm;
                    const double* hk = sg.host_of(dh) + (size_t)k * ldhd;
                    for (int jj = checked; jj <= j && !cl.conv; ++jj) {
                        double* hc = &cl.H[(size_t)jj * (J + 1)];
                        for (int i = 0; i <= jj + 1; ++i) hc[i] = hk[(size_t)jj * (J + 1) + i];
                        const double hn = hc[jj + 1];
                        for (int i = 0; i < jj; ++i) {
                            double t0 = cl.cs[i] * hc[i] + cl.sn[i] * hc[i + 1];
                            hc[i + 1] = -cl.sn[i] * hc[i] + cl.cs[i] * hc[i + 1];
                            hc[i] = t0;
                        }
                        double rr = std::hypot(hc[jj], hc[jj + 1]);
                        cl.cs[jj] = rr > 0 ? hc[jj] / rr : 1.0;
                        cl.sn[jj] = rr > 0 ? hc[jj + 1] / rr : 0.0;
                        hc[jj] = rr;
                        hc[jj + 1] = 0.0;
                        cl.g[jj + 1] = -cl.sn[jj] * cl.g[jj];
                        cl.g[jj] = cl.cs[jj] * cl.g[jj];
                        cl.used = jj + 1;
                        total++;
                        cl.conv = std::fabs(cl.g[jj + 1]) <= target || hn == 0.0;
                    }
                    all_conv = all_conv && cl.conv;
                }
                checked = j + 1;
            }
            // y = R^{-1} g per column, w += T y over that column's own steps
            bool done = true;
            GmSteps ju{};
            std::fill(ys.begin(), ys.end(), 0.0);
            for (int k = 0; k < m; ++k) {
                ColState& cl = cols[k];
                if (!cl.active || cl.used == 0) continue;
                const int jn = cl.used;
                for (int i = jn - 1; i >= 0; --i) {
                    double t0 = cl.g[i];
                    for (int q = i + 1; q < jn; ++q) t0 -= cl.H[(size_t)q * (J + 1) + i] * y[q];
                    y[i] = t0 / cl.H[(size_t)i * (J + 1) + i];
                }
                if constexpr (IR) {
                    ju.v[k] = jn;
                    for (int i = 0; i < jn; ++i) ys[(size_t)k * J + i] = y[i];
                } else {
                    double* dy;
                    ST_TRY(sg.in(y.data(), jn, &dy));
                    ST_TRY(st_tsgemm_nn(n, jn, 1, 1.0, T + (size_t)k * n, m * n, dy, jn, 1.0, Wg + (size_t)k * ldw,
                                        ldw, c.s));
                }
                done = done && cl.conv;
            }
            if constexpr (IR) {
                double* dys;
                ST_TRY(sg.in(ys.data(), (size_t)J * m, &dys));
                ST_TRY(st_gm_accumulate32(n, m, T, dys, J, ju, Wg, ldw, c.s));
                done = false;   // the FP32 cycle met its own target; the next cycle checks the FP64 residual
            }
            ST_TRY(sg.fetch());   // the upload region is reused by the next cycle
            if (done) break;
            // restart from the true residual R = B - (A + s M) W (FP64)
            double* Rd;
            if constexpr (IR)
                Rd = R;
            else
                Rd = Z;
            ST_TRY(st_spmm_comb64(p, -shift, -1.0, Wg, ldw, m, 0.0, Rd, n, c.s));
            ST_TRY(st_axpby64(n, m, 1.0, B, n, 1.0, Rd, n, c.s));
        }
    }
    if (iters_out) *iters_out += total;
    return ST_OK;
}

// FP32 iterative refinement for mixed precision where the work is bandwidth-
// or FP64-bound (at least 2^15 grid points, box stencils for the FP32 product);
// FP64 Krylov vectors otherwise.
int shifted_solve_fgmres(Ctx& c, int prec, double shift, const double* X, int ldx, const double* MX, int ldmx,
                         int ncols, double* W, int ldw, double rtol, int* iters_out) {
    const bool ir = prec == ST_MIXED && c.n >= (1 << 15) && c.p->box_ok && (c.p->dim == 2 || c.p->dim == 3);
    if (ir) return fgmres_impl<float>(c, prec, shift, X, ldx, MX, ldmx, ncols, W, ldw, rtol, iters_out);
    return fgmres_impl<double>(c, prec, shift, X, ldx, MX, ldmx, ncols, W, ldw, rtol, iters_out);
}

// RKSM driver.  Each iteration synchronises twice: after phase A (shifted
// solve, block CGS2 with its coefficients kept on the device, Gram matrices
// of the new block) and after phase B (CholQR2 finished on the device,
// products of the new block with V, MV, itself and F1).  Everything k x k
// runs on the host between the two.
int solve_impl(st_problem* p, const double* F1, int ldf1, const double* F2, int ldf2, int p0, st_solution* sol,
               st_stats* st) {
    hostpar::ActiveSolve active;   // solves in flight share the host cores
    auto t_start = Clock::now();
    Ctx c{p, p->stream, p->n_h};
    const int n = p->n_h, nt = p->n_t;
    const double dt = p->dt;
    // problems given as CSR matrices run in FP64 (the inner solver is FP64 CG)
    const int prec = p->dim == 0 ? ST_FP64 : p->d.precision;
    const double tol = p->d.tol;
    st_stats S{};
    auto tp = Clock::now();
    Stage sg(c);
    // heat: A symmetric, exact fast-diagonalisation shifted solves; convection-diffusion:
    // A nonsymmetric, preconditioned FGMRES shifted solves and unsymmetrised projections
    const bool sym = p->tensor_heat || p->dim == 0;
    if (p->dim == 0) ST_TRY(csr_spectrum(c));
    const double inner_tol = std::max(1e-13, 1e-3 * tol);
    auto resolvent = [&](double s, const double* X, int ldx, const double* MX, int ldmx, int m, double* W,
                         int ldw) -> int {
        if (sym) return shifted_solve(c, prec, s, X, ldx, MX, ldmx, m, W, ldw);
        return shifted_solve_fgmres(c, prec, s, X, ldx, MX, ldmx, m, W, ldw, inner_tol, &S.inner_iterations);
    };

    // ---- A1: rank compression of F = F1 F2^T ----
    double* F1d;
    ST_TRY(st_slot(p, S_F1D, sizeof(double) * (size_t)n * p0, (void**)&F1d));
    ST_TRY(st_stage_matrix(p, F1, ldf1, n, p0, F1d));
    const bool f2dev = st_is_device_ptr(F2);
    ST_TRY(stage_reserve(p, pad32((size_t)p0 * p0) + pad32((size_t)nt * p0)));
    double* dGF = sg.out((size_t)p0 * p0);
    ST_TRY(ts_tn_dev(c, p0, p0, F1d, n, F1d, n, dGF, p0));
    double* dF2 = nullptr;
    if (f2dev) {
        dF2 = sg.out((size_t)nt * p0);
        ST_CUDA_TRY(cudaMemcpy2DAsync(dF2, sizeof(double) * nt, F2, sizeof(double) * ldf2, sizeof(double) * nt, p0,
                                      cudaMemcpyDeviceToDevice, c.s));
    }
    ST_TRY(sg.fetch());
    std::vector<double> F2h((size_t)nt * p0);
    if (f2dev) {
        std::memcpy(F2h.data(), sg.host_of(dF2), sizeof(double) * (size_t)nt * p0);
    } else {
        for (int j = 0; j < p0; ++j) std::memcpy(&F2h[(size_t)j * nt], F2 + (size_t)j * ldf2, sizeof(double) * nt);
    }
    {
        // a NaN or Inf in F1 (seen through its Gram matrix) or F2 would make the kept rank 0
        // and the call return U = 0 as converged: refuse it instead
        const double* g = sg.host_of(dGF);
        bool finite = true;
        for (size_t i = 0; i < (size_t)p0 * p0; ++i) finite = finite && std::isfinite(g[i]);
        for (double v : F2h) finite = finite && std::isfinite(v);
        if (!finite) {
            st_note_msg("st_solve: F1 or F2 holds a NaN or Inf (or F1^T F1 overflows)");
            return ST_EINVAL;
        }
    }
    // F1 = Q1 R1 from F1^T F1 = E diag(w) E^T: Q1 = F1 E_r w_r^{-1/2}, R1 = w_r^{1/2} E_r^T
    // over the kept directions.  One Gram product loses orthogonality like
    // eps cond(F1)^2, so a condition number above 1e4 takes the CholQR2 route.
    std::vector<double> R1((size_t)p0 * p0, 0.0), T1;   // R1: r1 x p0 in a p0 x p0 array (ld p0)
    int r1 = 0, src_cols = 0;
    {
        std::vector<double> E(sg.host_of(dGF), sg.host_of(dGF) + (size_t)p0 * p0), w(p0);
        dense::sym_eig(p0, E.data(), p0, w.data());
        double wmax = std::max(w[p0 - 1], 0.0);
        for (int i = 0; i < p0; ++i) r1 += (wmax > 0.0 && w[i] > 1e-28 * wmax);
        bool gram = r1 > 0 && w[p0 - r1] > 1e-8 * wmax;
        if (gram) {
            T1.assign((size_t)p0 * r1, 0.0);
            for (int t = 0; t < r1; ++t) {
                int e = p0 - r1 + t;
                double sw = std::sqrt(w[e]);
                for (int q = 0; q < p0; ++q) {
                    R1[(size_t)q * p0 + t] = sw * E[(size_t)e * p0 + q];
                    T1[(size_t)t * p0 + q] = E[(size_t)e * p0 + q] / sw;
                }
            }
            src_cols = p0;
        } else if (r1 > 0) {
            ST_TRY(block_qr(c, F1d, n, p0, 0.0, 1e-14, R1, &r1));   // F1d <- Q1 (n x r1), F1 = Q1 R1
            T1.assign((size_t)r1 * r1, 0.0);
            for (int t = 0; t < r1; ++t) T1[(size_t)t * r1 + t] = 1.0;
            src_cols = r1;
        }
    }
    // F2 = Q2 R2 (host Householder)
    std::vector<double> Q2 = F2h, R2((size_t)p0 * p0);
    dense::thin_qr(nt, p0, Q2.data(), nt, R2.data(), p0);
    // B = R1 R2^T (r1 x p0)
    std::vector<double> B((size_t)r1 * p0, 0.0);
    for (int j = 0; j < p0; ++j)
        for (int i = 0; i < r1; ++i) {
            double s = 0.0;
            for (int q = 0; q < p0; ++q) s += R1[(size_t)q * p0 + i] * R2[(size_t)q * p0 + j];
            B[(size_t)j * r1 + i] = s;
        }
    int r = 0;
    std::vector<double> Ub, sb, Vbt;
    if (r1 > 0) {
        // SVD of B^T (p0 x r1): B = V2 diag(s2) U2^T
        std::vector<double> Bt((size_t)p0 * r1);
        for (int j = 0; j < p0; ++j)
            for (int i = 0; i < r1; ++i) Bt[(size_t)i * p0 + j] = B[(size_t)j * r1 + i];
        std::vector<double> U2((size_t)p0 * r1), s2(r1), V2t((size_t)r1 * r1);
        dense::svd_small(p0, r1, Bt.data(), p0, U2.data(), s2.data(), V2t.data());
        for (int i = 0; i < r1; ++i)
            if (s2[i] > 1e-14 * s2[0]) ++r;
        // F1c = Q1 V2[:, :r], F2c = Q2 U2[:, :r] diag(s)
        Ub.assign((size_t)r1 * r, 0.0);
        for (int j = 0; j < r; ++j)
            for (int i = 0; i < r1; ++i) Ub[(size_t)j * r1 + i] = V2t[(size_t)i * r1 + j];
        sb.assign(s2.begin(), s2.begin() + r);
        Vbt.assign((size_t)p0 * r, 0.0);
        for (int j = 0; j < r; ++j)
            for (int i = 0; i < p0; ++i) Vbt[(size_t)j * p0 + i] = U2[(size_t)j * p0 + i];
    }
    double normF = 0.0;
    for (double v : sb) normF += v * v;
    normF = std::sqrt(normF);
    S.p = r;
    if (r == 0) {
        // F = 0: U = 0
        p->k = 0;
        if (sol) {
            sol->n_h = n;
            sol->n_t = nt;
            sol->k = 0;
            sol->V = p->V;
            sol->Y = p->Y;
            if (sol->U_dense)
                for (int l = 0; l < nt; ++l)
                    ST_CUDA_TRY(cudaMemsetAsync(sol->U_dense + (size_t)l * sol->ldu, 0, sizeof(double) * n, c.s));
        }
        ST_CUDA_TRY(cudaStreamSynchronize(c.s));
        S.converged = 1;
        S.ms_total = ms_since(t_start);
        if (st) *st = S;
        return ST_OK;
    }
    double* F1c;
    ST_TRY(st_slot(p, S_F1C, sizeof(double) * (size_t)n * r, (void**)&F1c));
    {
        // F1c = source Tc with source = F1 (Gram route) or Q1 (CholQR2 route)
        std::vector<double> Tc((size_t)src_cols * r, 0.0);
        for (int j = 0; j < r; ++j)
            for (int t = 0; t < r1; ++t) {
                double u = Ub[(size_t)j * r1 + t];
                for (int q = 0; q < src_cols; ++q) Tc[(size_t)j * src_cols + q] += T1[(size_t)t * src_cols + q] * u;
            }
        ST_TRY(stage_reserve(p, pad32(Tc.size())));
        double* dTc;
        ST_TRY(sg.in(Tc.data(), Tc.size(), &dTc));
        ST_TRY(st_tsgemm_nn(n, src_cols, r, 1.0, F1d, n, dTc, src_cols, 0.0, F1c, n, c.s));
    }
    std::vector<double> F2c((size_t)nt * r, 0.0);   // Q2 U2 diag(s)
    for (int j = 0; j < r; ++j)
        for (int i = 0; i < nt; ++i) {
            double s = 0.0;
            for (int q = 0; q < p0; ++q) s += Q2[(size_t)q * nt + i] * Vbt[(size_t)j * p0 + q];
            F2c[(size_t)j * nt + i] = s * sb[j];
        }
    S.ms_phase[0] += ms_since(tp);

    // ---- start block v_1 = orth(M^{-1} F1c) ----
    const int pmax = r;
    double* MV = nullptr;
    ST_TRY(ensure_basis(p, c, std::min(2 * pmax + 8, p->d.max_basis + 16), 0, &MV));
    double* MAq;   // [M q, A q] staging, n x 2 pmax
    const int nmaq = sym ? 2 : 3;   // [M q, A q] or [M q, A q, A^T q]
    ST_TRY(st_slot(p, S_MAQ, sizeof(double) * (size_t)n * nmaq * pmax, (void**)&MAq));
    tp = Clock::now();
    ST_TRY(stage_reserve(p, 3 * pad32((size_t)r * r) + pad32(1) + pad32((size_t)2 * r * r) + pad32((size_t)r * r)));
    ST_TRY(mass_inverse(c, prec, F1c, n, r, p->V, n));
    double* dG = sg.out((size_t)r * r);
    ST_TRY(ts_tn_dev(c, r, r, p->V, n, p->V, n, dG, r));
    ST_TRY(sg.fetch());
    S.ms_phase[1] += ms_since(tp);
    tp = Clock::now();
    int k = 0;
    double* dflag = nullptr;
    {
        QrPlan qp;
        qr_plan(sg.host_of(dG), r, 0.0, 1e-12, qp);
        if (qp.rank == 0) return breakdown("start block has rank 0");
        if (qp.fast) {
            double* dR2;
            ST_TRY(qr_fast_launch(c, sg, p->V, n, r, qp.R1, &dR2, &dflag));
            k = r;
        } else {
            std::vector<double> Rx;
            ST_TRY(block_qr(c, p->V, n, r, 0.0, 1e-12, Rx, &k));
            if (k == 0) return breakdown("start block has rank 0");
        }
    }
    const bool dfb = prec == ST_MIXED;
    if (dfb) ST_TRY(st_to_df(n, k, p->V, n, p->Vdf, n, c.s));
    ST_TRY(st_spmm_ma<double>(p, p->V, n, k, MAq, n, MAq + (size_t)n * k, n, c.s));
    double* dX0 = sg.out((size_t)k * 2 * k);
    ST_TRY(ts_tn_dev(c, k, 2 * k, p->V, n, MAq, n, dX0, k));
    double* dG1 = sg.out((size_t)k * r);
    ST_TRY(ts_tn_dev(c, k, r, p->V, n, F1c, n, dG1, k));
    ST_CUDA_TRY(cudaMemcpyAsync(MV, MAq, sizeof(double) * (size_t)n * k, cudaMemcpyDeviceToDevice, c.s));
    ST_TRY(sg.fetch());
    if (dflag && sg.host_of(dflag)[0] != 0.0) return breakdown("start block: device Cholesky pivot not positive");
    HostSym Mm, Am, Hb;
    std::vector<double> Gm;   // k x r, ld = ldg
    int ldg = 0;
    {
        const double* X = sg.host_of(dX0);
        const double* G = sg.host_of(dG1);
        Mm.grow(k);
        Am.grow(k);
        for (int j = 0; j < k; ++j)
            for (int i = 0; i < k; ++i) {
                Mm(i, j) = 0.5 * (X[(size_t)j * k + i] + X[(size_t)i * k + j]);
                Am(i, j) = sym ? 0.5 * (X[(size_t)(k + j) * k + i] + X[(size_t)(k + i) * k + j])
                               : X[(size_t)(k + j) * k + i];
            }
        ldg = std::max(64, 2 * k);
        Gm.assign((size_t)ldg * r, 0.0);
        for (int j = 0; j < r; ++j)
            for (int i = 0; i < k; ++i) Gm[(size_t)j * ldg + i] = G[(size_t)j * k + i];
    }
    S.ms_phase[3] += ms_since(tp);
    std::vector<int> boff{0}, bsz{k};
    std::vector<double> shifts, ritz, Y;
    int last_ritz_k = -1;
    double res = 1.0;
    int status = ST_ENOTCONV;
    int it = 0;
    int next_check = 1;
    int mu_extra = 0;
    const double a_int = p->lam_min, b_int = p->lam_max;
    std::vector<int> hist_it;
    std::vector<double> hist_res;

    while (true) {
        if (it >= p->d.maxit) break;
        const int pl = bsz.back();
        const int lo = boff.back();
        if (k + pl > p->d.max_basis) break;
        ST_TRY(ensure_basis(p, c, k + pl, k, &MV));
        // ---- shift ----
        tp = Clock::now();
        // Ritz values cost O(k^3) on the host: refresh them while the basis is
        // small, then whenever it has grown by an eighth (a quarter beyond 64
        // columns) since the last refresh
        if (last_ritz_k < 0 || k <= 16 ||
            k >= last_ritz_k + std::max(2, last_ritz_k / (last_ritz_k > 64 ? 4 : 8))) {
            if (!ritz_values(k, Am.a.data(), Mm.a.data(), Mm.ld, ritz)) ritz.clear();
            last_ritz_k = k;
        }
        double s = next_shift(a_int, b_int, shifts, ritz, 80);
        shifts.push_back(s);
        S.ms_phase[7] += ms_since(tp);
        ++it;
        size_t needA = 2 * pad32((size_t)(k + pl) * pl);
        size_t needB = pad32((size_t)(k + pl) * nmaq * pl) + pad32((size_t)pl * r) + 2 * pad32((size_t)pl * pl) +
                       pad32(1);
        ST_TRY(stage_reserve(p, std::max(needA, needB)));
        // ---- phase A: A3 shifted solve into the next basis slot, A4 block CGS2 ----
        tp = Clock::now();
        double* W = p->V + (size_t)k * n;
        ST_TRY(resolvent(s, p->V + (size_t)lo * n, n, MV + (size_t)lo * n, n, pl, W, n));
        // each pass is one product [V, W]^T W: its first k rows are the Gram-Schmidt
        // coefficients, its last pl rows the Gram matrix of W before the update.  Mixed
        // precision: the first pass in FP32 on the leading parts, the second in double-float
        // (the update W - V h of both passes in double-float, so W = V (h0 + h1) + W' holds
        // to double-float accuracy whatever the accuracy of h0)
        const int kk = k + pl;
        double* dh[2];
        for (int pass = 0; pass < 2; ++pass) {
            dh[pass] = sg.out((size_t)kk * pl);
            if (dfb) {
                ST_TRY(st_to_df(n, pl, W, n, p->Vdf + (size_t)k * n, n, c.s));
                double* part;
                ST_TRY(st_slot(p, S_PART, sizeof(double) * st_tsgemm_partial_elems(n, kk, pl), (void**)&part));
                ST_TRY(st_tsgemm_tn_df(n, kk, pl, p->Vdf, n, p->Vdf + (size_t)k * n, n, dh[pass], kk, part, c.s,
                                       pass == 0));
            } else {
                ST_TRY(ts_tn_dev(c, kk, pl, p->V, n, W, n, dh[pass], kk));
            }
            ST_TRY(basis_nn_sub(c, dfb, k, pl, dh[pass], kk, W, n));
        }
        ST_TRY(sg.fetch());
        S.ms_phase[1] += ms_since(tp);
        tp = Clock::now();
        std::vector<double> Hcol((size_t)k * pl), Gw((size_t)pl * pl);
        double ref2 = 0.0, tr1 = 0.0, tr2 = 0.0;
        {
            const double* h0 = sg.host_of(dh[0]);
            const double* h1 = sg.host_of(dh[1]);
            for (int j = 0; j < pl; ++j)
                for (int i = 0; i < k; ++i) Hcol[(size_t)j * k + i] = h0[(size_t)j * kk + i] + h1[(size_t)j * kk + i];
            // Gram of W after the second pass: G1 - h2^T h2 (V orthonormal), G1 the Gram before it
            for (int j = 0; j < pl; ++j) {
                ref2 = std::max(ref2, h0[(size_t)j * kk + k + j]);
                for (int i = 0; i < pl; ++i) {
                    double g = h1[(size_t)j * kk + k + i], hh = 0.0;
                    for (int q = 0; q < k; ++q) hh += h1[(size_t)i * kk + q] * h1[(size_t)j * kk + q];
                    Gw[(size_t)j * pl + i] = g - hh;
                    if (i == j) {
                        tr1 += g;
                        tr2 += hh;
                    }
                }
            }
        }
        if (!(tr2 <= 1e-4 * tr1)) {
            // the second pass removed a visible part: take the Gram matrix explicitly
            ST_TRY(ts_tn_host(c, pl, pl, W, n, W, n, Gw.data()));
        }
        QrPlan qp;
        qr_plan(Gw.data(), pl, ref2, 1e-10, qp);
        if (qp.severe) {
            // the block almost lies in range(V): its remainder carries the rounding
            // of the two passes, so a third pass in FP64 cleans it before the QR
            std::vector<double> h3((size_t)k * pl), G3((size_t)pl * pl);
            ST_TRY(ts_tn_host(c, k, pl, p->V, n, W, n, h3.data()));
            ST_TRY(ts_nn_host(c, k, pl, -1.0, p->V, n, h3.data(), 1.0, W, n));
            for (size_t i = 0; i < Hcol.size(); ++i) Hcol[i] += h3[i];
            ST_TRY(ts_tn_host(c, pl, pl, W, n, W, n, G3.data()));
            qr_plan(G3.data(), pl, ref2, 1e-10, qp);
        }
        int pn = 0;
        std::vector<double> Rq((size_t)pl * pl, 0.0);
        double* dR2 = nullptr;
        dflag = nullptr;
        if (qp.rank > 0) {
            if (qp.fast) {
                ST_TRY(qr_fast_launch(c, sg, W, n, pl, qp.R1, &dR2, &dflag));
                pn = pl;
            } else {
                ST_TRY(block_qr(c, W, n, pl, ref2, 1e-10, Rq, &pn));
            }
        }
        S.ms_phase[2] += ms_since(tp);
        // ---- phase B: A5 products of the new block ----
        tp = Clock::now();
        std::vector<double> X1, X2, X3;
        if (pn > 0) {
            ST_TRY(st_spmm_ma<double>(p, W, n, pn, MAq, n, MAq + (size_t)n * pn, n, c.s));
            if (!sym) ST_TRY(st_spmm_at64(p, W, n, pn, MAq + (size_t)2 * n * pn, n, c.s));
            if (dfb) ST_TRY(st_to_df(n, pn, W, n, p->Vdf + (size_t)k * n, n, c.s));
            // one product [V, q]^T [M q, A q (, A^T q)]: rows 0..k-1 = V^T (.), rows k.. = q^T (.)
            const int kq = k + pn;
            double* dX12 = sg.out((size_t)kq * nmaq * pn);
            ST_TRY(basis_tn(c, dfb, kq, nmaq * pn, MAq, n, dX12, kq));
            double* dX3 = sg.out((size_t)pn * r);
            ST_TRY(ts_tn_dev(c, pn, r, W, n, F1c, n, dX3, pn));
            ST_TRY(sg.fetch());
            if (qp.fast) {
                if (sg.host_of(dflag)[0] != 0.0) return breakdown("new block: device Cholesky pivot not positive");
                Rq = upper_product(pl, sg.host_of(dR2), qp.R1.data());
            }
            auto grab = [&](const double* d, size_t m) { return std::vector<double>(sg.host_of(d), sg.host_of(d) + m); };
            {
                const double* x12 = sg.host_of(dX12);
                X1.resize((size_t)k * nmaq * pn);
                X2.resize((size_t)pn * 2 * pn);
                for (int j = 0; j < nmaq * pn; ++j)
                    for (int i = 0; i < k; ++i) X1[(size_t)j * k + i] = x12[(size_t)j * kq + i];
                for (int j = 0; j < 2 * pn; ++j)
                    for (int i = 0; i < pn; ++i) X2[(size_t)j * pn + i] = x12[(size_t)j * kq + k + i];
            }
            X3 = grab(dX3, (size_t)pn * r);
        }
        S.ms_phase[3] += ms_since(tp);
        mu_extra = pn;
        // Hbar column block: rows 0..k-1 = Hcol, rows k..k+pn-1 = Rq
        Hb.grow(k + pn);
        for (int j = 0; j < pl; ++j) {
            for (int i = 0; i < k; ++i) Hb(i, lo + j) = Hcol[(size_t)j * k + i];
            for (int i = 0; i < pn; ++i) Hb(k + i, lo + j) = Rq[(size_t)j * pl + i];
        }
        // ---- A6/A7 residual check of the current basis V (k columns) ----
        bool check = (pn == 0) || (it >= next_check) || (it >= p->d.maxit) || (k + pn + pn > p->d.max_basis);
        if (check) {
            tp = Clock::now();
            if (!projected_solve(k, nt, dt, Mm.a.data(), Am.a.data(), Mm.ld, Gm.data(), ldg, r, F2c.data(), Y, sym))
                return breakdown("projected equation singular");
            S.ms_phase[4] += ms_since(tp);
            S.residual_checks++;
            tp = Clock::now();
            double rr = 0.0;
            if (pn > 0) {
                std::vector<double> Gb;
                ST_TRY(residual_gram_explicit(c, k, pn, pl, s, MAq, MV, X1, Mm, Rq, Gb));
                // f = H^{-T} E_last  (k x pl)
                std::vector<double> H((size_t)k * k), f((size_t)k * pl, 0.0);
                for (int j = 0; j < k; ++j)
                    for (int i = 0; i < k; ++i) H[(size_t)j * k + i] = Hb(i, j);
                std::vector<int> piv(k);
                dense::lu(k, H.data(), k, piv.data());
                for (int j = 0; j < pl; ++j) f[(size_t)j * k + lo + j] = 1.0;
                if (!dense::lu_solve_transpose(k, H.data(), k, piv.data(), f.data(), k, pl)) return breakdown("rational Arnoldi Hessenberg matrix singular");
                // g_l = f^T (dt/2)(y_l + y_{l-1});  ||R||^2 = sum_l g_l^T Gb g_l
                std::vector<double> gl(pl);
                for (int l = 0; l < nt; ++l) {
                    const double* y = &Y[(size_t)l * k];
                    const double* yp = l > 0 ? &Y[(size_t)(l - 1) * k] : nullptr;
                    for (int j = 0; j < pl; ++j) {
                        double sacc = 0.0;
                        const double* fj = &f[(size_t)j * k];
                        for (int i = 0; i < k; ++i) sacc += fj[i] * (y[i] + (yp ? yp[i] : 0.0));
                        gl[j] = 0.5 * dt * sacc;
                    }
                    for (int a = 0; a < pl; ++a)
                        for (int b2 = 0; b2 < pl; ++b2) rr += gl[a] * Gb[(size_t)b2 * pl + a] * gl[b2];
                }
            }
            res = std::sqrt(std::max(rr, 0.0)) / normF;
            S.ms_phase[5] += ms_since(tp);
            if (res <= tol || pn == 0) {
                status = res <= tol ? ST_OK : ST_ENOTCONV;
                if (pn == 0 && res > tol) status = ST_EBREAKDOWN;
                break;
            }
            next_check = it + check_gap(hist_it, hist_res, it, res, tol, (double)k * k * nt);
            hist_it.push_back(it);
            hist_res.push_back(res);
        }
        if (pn == 0) {
            status = ST_EBREAKDOWN;
            break;
        }
        // ---- append the new block ----
        tp = Clock::now();
        ST_CUDA_TRY(cudaMemcpyAsync(MV + (size_t)k * n, MAq, sizeof(double) * (size_t)n * pn, cudaMemcpyDeviceToDevice,
                                    c.s));
        const int kn = k + pn;
        Mm.grow(kn);
        Am.grow(kn);
        for (int j = 0; j < pn; ++j) {
            for (int i = 0; i < k; ++i) {
                Mm(i, k + j) = Mm(k + j, i) = X1[(size_t)j * k + i];
                Am(i, k + j) = X1[(size_t)(pn + j) * k + i];
                Am(k + j, i) = sym ? X1[(size_t)(pn + j) * k + i] : X1[(size_t)(2 * pn + j) * k + i];
            }
            for (int i = 0; i < pn; ++i) {
                Mm(k + i, k + j) = 0.5 * (X2[(size_t)j * pn + i] + X2[(size_t)i * pn + j]);
                Am(k + i, k + j) = sym ? 0.5 * (X2[(size_t)(pn + j) * pn + i] + X2[(size_t)(pn + i) * pn + j])
                                       : X2[(size_t)(pn + j) * pn + i];
            }
        }
        if (kn > ldg) {
            int nl = std::max(2 * ldg, kn);
            std::vector<double> g2((size_t)nl * r, 0.0);
            for (int j = 0; j < r; ++j)
                for (int i = 0; i < k; ++i) g2[(size_t)j * nl + i] = Gm[(size_t)j * ldg + i];
            Gm.swap(g2);
            ldg = nl;
        }
        for (int j = 0; j < r; ++j)
            for (int i = 0; i < pn; ++i) Gm[(size_t)j * ldg + k + i] = X3[(size_t)j * pn + i];
        boff.push_back(k);
        bsz.push_back(pn);
        k = kn;
        S.ms_phase[3] += ms_since(tp);
    }
    if (Y.empty() || (int)(Y.size() / std::max(1, nt)) != k) {
        // iterations ended without a check of the final basis
        if (!projected_solve(k, nt, dt, Mm.a.data(), Am.a.data(), Mm.ld, Gm.data(), ldg, r, F2c.data(), Y, sym))
            return breakdown("projected equation singular (final basis)");
        mu_extra = 0;
    }
    // ---- A9 output ----
    tp = Clock::now();
    if (p->Y_cap < (size_t)k * nt) {
        if (p->Y) st_free_one(p, p->Y);
        p->Y = nullptr;
        p->Y_cap = 0;
        ST_TRY(st_alloc(p, (void**)&p->Y, sizeof(double) * (size_t)k * nt));
        p->Y_cap = (size_t)k * nt;
    }
    ST_TRY(write_dev(c, Y.data(), k, k, nt, p->Y, k));
    p->k = k;
    if (sol) {
        sol->n_h = n;
        sol->n_t = nt;
        sol->k = k;
        sol->V = p->V;
        sol->Y = p->Y;
        if (sol->U_dense) {
            if (sol->ldu < n) return ST_EINVAL;
            ST_TRY(st_lowrank_dense(n, k, nt, p->V, n, p->Y, k, sol->U_dense, sol->ldu, c.s));
        }
    }
    ST_CUDA_TRY(cudaStreamSynchronize(c.s));
    S.ms_phase[6] += ms_since(tp);
    // numerical rank of Y (V orthonormal): eigenvalues of Y Y^T
    if (st) {
        std::vector<double> G((size_t)k * k, 0.0), w(k);
        for (int l = 0; l < nt; ++l) {
            const double* y = &Y[(size_t)l * k];
            for (int j = 0; j < k; ++j)
                for (int i = 0; i <= j; ++i) G[(size_t)j * k + i] += y[i] * y[j];
        }
        for (int j = 0; j < k; ++j)
            for (int i = j + 1; i < k; ++i) G[(size_t)j * k + i] = G[(size_t)i * k + j];
        dense::sym_eigvals(k, G.data(), k, w.data());
        double smax = k ? std::sqrt(std::max(w[k - 1], 0.0)) : 0.0;
        int rank = 0;
        for (int i = 0; i < k; ++i) rank += std::sqrt(std::max(w[i], 0.0)) > 1e-8 * smax;
        S.rank = rank;
    }
    S.iterations = it;
    S.basis_cols = k;
    S.mu_mem = k + mu_extra;
    S.relres = res;
    S.converged = res <= tol;
    if (!shifts.empty()) {
        S.shift_min = *std::min_element(shifts.begin(), shifts.end());
        S.shift_max = *std::max_element(shifts.begin(), shifts.end());
    }
    S.ms_total = ms_since(t_start);
    if (st) *st = S;
    if (status == ST_EBREAKDOWN && res <= tol) status = ST_OK;
    return status;
}

// ||L Z^T||_F for L (device n x m, overwritten) and Z (host nt x m): QR of L one
// column at a time, then the small product R Z^T on the host.  The factor
// [F1, M V, A V] of a residual is far from full rank (F1 lies in range(M V),
// A V mostly in range(M V) too) and its columns differ in norm by orders of
// magnitude, so each column is re-projected until a pass no longer halves it
// ("twice is enough" made adaptive, at most four passes), and a column whose
// remainder falls below 1e-13 of its original norm adds no direction.  This
// keeps the backward error per column near rounding, like a Householder QR.
int lowrank_fro(Ctx& c, double* L, int m, const std::vector<double>& Z, int nt, double* out) {
    const int n = c.n;
    std::vector<double> R((size_t)m * m, 0.0);
    int q = 0;
    std::vector<double> nu2(1), h;
    for (int j = 0; j < m; ++j) {
        double* w = L + (size_t)j * n;
        ST_TRY(ts_tn_host(c, 1, 1, w, n, w, n, nu2.data()));
        const double nu0 = std::sqrt(std::max(nu2[0], 0.0));
        double nu = nu0;
        std::vector<double> coef((size_t)std::max(q, 1), 0.0);
        for (int pass = 0; pass < 4 && q > 0 && nu > 0.0; ++pass) {
            h.assign(q, 0.0);
            ST_TRY(ts_tn_host(c, q, 1, L, n, w, n, h.data()));
            ST_TRY(ts_nn_host(c, q, 1, -1.0, L, n, h.data(), 1.0, w, n));
            for (int i = 0; i < q; ++i) coef[i] += h[i];
            ST_TRY(ts_tn_host(c, 1, 1, w, n, w, n, nu2.data()));
            double nu_new = std::sqrt(std::max(nu2[0], 0.0));
            bool settled = nu_new > 0.5 * nu;
            nu = nu_new;
            if (settled) break;
        }
        for (int i = 0; i < q; ++i) R[(size_t)j * m + i] = coef[i];
        if (nu > 1e-13 * nu0 && nu > 0.0) {
            double* dst = L + (size_t)q * n;
            ST_TRY(st_axpby64(n, 1, 1.0 / nu, w, n, 0.0, dst, n, c.s));
            R[(size_t)j * m + q] = nu;
            ++q;
        }
    }
    double s = 0.0;
    for (int l = 0; l < nt; ++l)
        for (int i = 0; i < q; ++i) {
            double v = 0.0;
            for (int j = 0; j < m; ++j) v += R[(size_t)j * m + i] * Z[(size_t)j * nt + l];
            s += v * v;
        }
    *out = std::sqrt(s);
    return ST_OK;
}

__global__ void k_dense_resid(int n, int nt, const double* __restrict__ F1, long long ldf1,
                              const double* __restrict__ F2, long long ldf2, int p, const double* __restrict__ Yop,
                              long long ldy, double* __restrict__ part) {
    __shared__ double sr[256], sf[256];
    double ar = 0.0, af = 0.0;
    long long tot = (long long)n * nt;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < tot;
         idx += (long long)gridDim.x * blockDim.x) {
        int l = (int)(idx / n), i = (int)(idx % n);
        double f = 0.0;
        for (int q = 0; q < p; ++q) f += F1[(size_t)q * ldf1 + i] * F2[(size_t)q * ldf2 + l];
        double rres = f - Yop[(size_t)l * ldy + i];
        ar += rres * rres;
        af += f * f;
    }
    sr[threadIdx.x] = ar;
    sf[threadIdx.x] = af;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sr[threadIdx.x] += sr[threadIdx.x + w];
            sf[threadIdx.x] += sf[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = sr[0];
        part[2 * blockIdx.x + 1] = sf[0];
    }
}

}  // namespace rksm

using namespace rksm;

extern "C" int st_solve(st_problem* p, const double* F1, int ldf1, const double* F2, int ldf2, int ncols,
                        st_solution* sol, st_stats* stats) {
    if (!p || !F1 || !F2) return ST_EINVAL;
    if (ncols < 1 || ncols > 16 || ldf1 < p->n_h || ldf2 < p->n_t) return ST_EINVAL;
    // box grids (heat or convection-diffusion); CSR matrices for heat (M and A symmetric positive definite)
    if (p->dim < 0 || (p->dim == 0 && p->d.op != ST_HEAT)) return ST_ENOTSUP;
    return solve_impl(p, F1, ldf1, F2, ldf2, ncols, sol, stats);
}

extern "C" int st_apply(st_problem* p, int dtype, const void* U, int ldu, void* Y, int ldy) {
    if (!p || !U || !Y || ldu < p->n_h || ldy < p->n_h) return ST_EINVAL;
    if (dtype == ST_F64) return st_apply_kernel<double>(p, (const double*)U, ldu, (double*)Y, ldy, p->n_t, p->stream);
    if (dtype == ST_F32) return st_apply_kernel<float>(p, (const float*)U, ldu, (float*)Y, ldy, p->n_t, p->stream);
    return ST_EINVAL;
}

extern "C" int st_shift_solve(st_problem* p, double s, const double* X, int ldx, int ncols, double* W, int ldw,
                              int precision) {
    if (!p || !X || !W || ncols < 1 || ldx < p->n_h || ldw < p->n_h) return ST_EINVAL;
    if (precision != ST_FP64 && precision != ST_MIXED) return ST_EINVAL;
    if (!p->tensor_heat && !(p->dim >= 1 && p->d.op == ST_CONVDIFF) && !(p->dim == 0 && p->d.op == ST_HEAT))
        return ST_ENOTSUP;
    if (!(s > -p->lam_min)) return ST_EINVAL;
    Ctx c{p, p->stream, p->n_h};
    // process in column groups of at most 16 through a private buffer (X and W may alias)
    for (int j0 = 0; j0 < ncols; j0 += 16) {
        int m = std::min(16, ncols - j0);
        double* buf;
        ST_TRY(st_slot(p, S_COPY, sizeof(double) * (size_t)p->n_h * m, (void**)&buf));
        if (p->tensor_heat || p->dim == 0)
            ST_TRY(shifted_solve(c, precision, s, X + (size_t)j0 * ldx, ldx, nullptr, 0, m, buf, p->n_h));
        else
            ST_TRY(shifted_solve_fgmres(c, precision, s, X + (size_t)j0 * ldx, ldx, nullptr, 0, m, buf, p->n_h, 1e-12,
                                        nullptr));
        ST_TRY(st_copy_cols64(p->n_h, m, buf, p->n_h, W + (size_t)j0 * ldw, ldw, p->stream));
    }
    return ST_OK;
}

extern "C" int st_autotune(st_problem* p, double s, int ncols, int precision, int* tuned) {
    if (tuned) *tuned = 0;
    if (!p || ncols < 1 || ncols > 16) return ST_EINVAL;
    if (precision != ST_FP64 && precision != ST_MIXED) return ST_EINVAL;
    if (!p->tensor_heat && !(p->dim >= 1 && p->d.op == ST_CONVDIFF)) return ST_ENOTSUP;
    if (!(s > -p->lam_min)) return ST_EINVAL;
    const size_t n = (size_t)p->n_h, bytes = sizeof(double) * n * (size_t)ncols;
    // seeded values in [-1, 1) from an integer hash: the solve must do real work (a
    // zero right-hand side would stop FGMRES before its first preconditioner call)
    std::vector<double> h(n * (size_t)ncols);
    for (size_t e = 0; e < h.size(); ++e) {
        uint32_t x = (uint32_t)e * 2654435761u + 0x9e3779b9u;
        x ^= x >> 15;
        x *= 0x85ebca6bu;
        x ^= x >> 13;
        h[e] = (double)(x >> 8) / 8388608.0 - 1.0;
    }
    double *X = nullptr, *W = nullptr;
    void* scratch = nullptr;
    int rc = ST_OK;
    if (cudaMalloc(&X, bytes) != cudaSuccess || cudaMalloc(&W, bytes) != cudaSuccess ||
        cudaMalloc(&scratch, bytes) != cudaSuccess) {
        cudaGetLastError();   // a failed allocation must not surface at a later launch check
        st_note_msg("st_autotune: device allocation failed");
        rc = ST_ENOMEM;
    }
    if (rc == ST_OK && cudaMemcpy(X, h.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) rc = ST_ECUDA;
    if (rc == ST_OK) {
        StTuneSession sess;
        sess.scratch = scratch;
        sess.scratch_bytes = bytes;
        st_tune_set_session(&sess);
        rc = st_shift_solve(p, s, X, (int)n, ncols, W, (int)n, precision);
        st_tune_set_session(nullptr);
        if (cudaStreamSynchronize(p->stream) != cudaSuccess && rc == ST_OK) rc = ST_ECUDA;
        if (tuned) *tuned = sess.tuned;
    }
    cudaFree(X);
    cudaFree(W);
    cudaFree(scratch);
    return rc;
}

extern "C" int st_autotune_reset(void) {
    sttune::table().clear();
    return ST_OK;
}

extern "C" int st_autotune_count(void) { return sttune::table().size(); }

// Tuning cache file (text): "st-autotune 1", "device <tag>", then one line
// "family tsize a b c d choice" per entry, sorted.
namespace {
bool valid_tag(const char* tag) {
    if (!tag || !*tag) return false;
    size_t n = 0;
    for (const char* c = tag; *c; ++c, ++n)
        if (*c == '\n' || *c == '\r') return false;
    return n < 200;
}
}  // namespace

extern "C" int st_autotune_save(const char* path, const char* device_tag) {
    if (!path || !valid_tag(device_tag)) return ST_EINVAL;
    std::vector<std::array<int, 7>> rows;
    sttune::table().for_each([&](const sttune::Key& k, int v) {
        rows.push_back({k.family, k.tsize, k.a, k.b, k.c, k.d, v});
    });
    std::sort(rows.begin(), rows.end());
    FILE* f = std::fopen(path, "w");
    if (!f) {
        st_note_msg("st_autotune_save: cannot open the file for writing");
        return ST_EINVAL;
    }
    bool ok = std::fprintf(f, "st-autotune 1\ndevice %s\n", device_tag) > 0;
    for (const auto& r : rows)
        ok = ok && std::fprintf(f, "%d %d %d %d %d %d %d\n", r[0], r[1], r[2], r[3], r[4], r[5], r[6]) > 0;
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) st_note_msg("st_autotune_save: write failed");
    return ok ? ST_OK : ST_EINVAL;
}

extern "C" int st_autotune_load(const char* path, const char* device_tag, int* loaded) {
    if (loaded) *loaded = 0;
    if (!path || !valid_tag(device_tag)) return ST_EINVAL;
    FILE* f = std::fopen(path, "r");
    if (!f) {
        st_note_msg("st_autotune_load: cannot open the file");
        return ST_EINVAL;
    }
    char line[512];
    auto next = [&]() -> bool {
        if (!std::fgets(line, sizeof(line), f)) return false;
        size_t n = std::strlen(line);
        while (n > 0 && (line[n - 1] == '\n' || line[n - 1] == '\r')) line[--n] = '\0';
        return true;
    };
    int rc = ST_OK;
    std::vector<std::pair<sttune::Key, int>> rows;
    if (!next() || std::strcmp(line, "st-autotune 1") != 0 || !next() || std::strncmp(line, "device ", 7) != 0) {
        st_note_msg("st_autotune_load: not a tuning cache (header)");
        rc = ST_EINVAL;
    } else if (std::strcmp(line + 7, device_tag) != 0) {
        st_note_msg("st_autotune_load: the cache was written for another device; nothing loaded");
    } else {
        while (next()) {
            if (line[0] == '\0') continue;
            int v[7];
            char extra;
            if (std::sscanf(line, "%d %d %d %d %d %d %d %c", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5], &v[6],
                            &extra) != 7) {
                st_note_msg("st_autotune_load: malformed entry; nothing loaded");
                rc = ST_EINVAL;
                break;
            }
            const sttune::Key k{v[0], v[1], v[2], v[3], v[4], v[5]};
            if (sttune::plausible(k, v[6])) rows.push_back({k, v[6]});
        }
    }
    std::fclose(f);
    if (rc != ST_OK) return rc;
    // a loaded choice is still checked against its launch's shape before use
    for (const auto& r : rows) sttune::table().put(r.first, r.second);
    if (loaded) *loaded = (int)rows.size();
    return ST_OK;
}

extern "C" int st_residual(st_problem* p, const double* U, int ldu, const double* F1, int ldf1, const double* F2,
                           int ldf2, int ncols, double* relres) {
    if (!p || !U || !F1 || !F2 || !relres || ncols < 1 || ldu < p->n_h || ldf1 < p->n_h || ldf2 < p->n_t)
        return ST_EINVAL;
    int n = p->n_h, nt = p->n_t;
    double *f1, *f2, *Yop, *part;
    ST_TRY(st_slot(p, S_LRQ, sizeof(double) * (size_t)n * ncols, (void**)&f1));
    ST_TRY(st_slot(p, S_LRZ, sizeof(double) * (size_t)nt * ncols, (void**)&f2));
    ST_TRY(st_slot(p, S_RES, sizeof(double) * (size_t)n * nt, (void**)&Yop));
    const int blocks = 1216;
    ST_TRY(st_slot(p, S_RESP, sizeof(double) * 2 * blocks, (void**)&part));
    ST_TRY(st_stage_matrix(p, F1, ldf1, n, ncols, f1));
    ST_TRY(st_stage_matrix(p, F2, ldf2, nt, ncols, f2));
    ST_TRY(st_apply_kernel<double>(p, U, ldu, Yop, n, nt, p->stream));
    k_dense_resid<<<blocks, 256, 0, p->stream>>>(n, nt, f1, n, f2, nt, ncols, Yop, n, part);
    ST_LAUNCH_CHECK();
    std::vector<double> h(2 * blocks);
    ST_CUDA_TRY(cudaMemcpyAsync(h.data(), part, sizeof(double) * 2 * blocks, cudaMemcpyDeviceToHost, p->stream));
    ST_CUDA_TRY(cudaStreamSynchronize(p->stream));
    double rr = 0.0, ff = 0.0;
    for (int b = 0; b < blocks; ++b) {
        rr += h[2 * b];
        ff += h[2 * b + 1];
    }
    *relres = ff > 0 ? std::sqrt(rr / ff) : std::sqrt(rr);
    return ST_OK;
}

extern "C" int st_residual_lowrank(st_problem* p, const double* V, int ldv, const double* Y, int ldy, int k,
                                   const double* F1, int ldf1, const double* F2, int ldf2, int ncols,
                                   double* relres) {
    if (!p || !V || !Y || !F1 || !F2 || !relres || k < 0 || ncols < 1 || ldv < p->n_h || ldy < std::max(1, k) ||
        ldf1 < p->n_h || ldf2 < p->n_t)
        return ST_EINVAL;
    Ctx c{p, p->stream, p->n_h};
    int n = p->n_h, nt = p->n_t;
    int m = ncols + 2 * k;
    double* L;
    ST_TRY(st_slot(p, S_LRQ, sizeof(double) * (size_t)n * m, (void**)&L));
    ST_TRY(st_stage_matrix(p, F1, ldf1, n, ncols, L));
    if (k > 0) ST_TRY(st_spmm_ma<double>(p, V, ldv, k, L + (size_t)n * ncols, n, L + (size_t)n * (ncols + k), n, c.s));
    // Z = [F2, -D_t Y^T, -C_t Y^T] on the host
    std::vector<double> Yh((size_t)std::max(1, k) * nt), F2h((size_t)nt * ncols);
    if (k > 0) ST_TRY(read_dev(c, Y, ldy, k, nt, Yh.data(), k));
    if (st_is_device_ptr(F2)) {
        ST_TRY(read_dev(c, F2, ldf2, nt, ncols, F2h.data(), nt));
    } else {
        for (int j = 0; j < ncols; ++j) std::memcpy(&F2h[(size_t)j * nt], F2 + (size_t)j * ldf2, sizeof(double) * nt);
    }
    std::vector<double> Z((size_t)nt * m, 0.0);
    for (int j = 0; j < ncols; ++j) std::memcpy(&Z[(size_t)j * nt], &F2h[(size_t)j * nt], sizeof(double) * nt);
    for (int a = 0; a < k; ++a)
        for (int l = 0; l < nt; ++l) {
            double y = Yh[(size_t)l * k + a], yp = l > 0 ? Yh[(size_t)(l - 1) * k + a] : 0.0;
            Z[(size_t)(ncols + a) * nt + l] = -(y - yp);
            Z[(size_t)(ncols + k + a) * nt + l] = -0.5 * p->dt * (y + yp);
        }
    double num = 0.0, den = 0.0;
    ST_TRY(lowrank_fro(c, L, m, Z, nt, &num));
    // ||F||: QR of F1 alone
    ST_TRY(st_stage_matrix(p, F1, ldf1, n, ncols, L));
    std::vector<double> Zf(F2h);
    ST_TRY(lowrank_fro(c, L, ncols, Zf, nt, &den));
    *relres = den > 0 ? num / den : num;
    return ST_OK;
}
