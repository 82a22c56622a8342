// Host side of the RKSM driver (paper Section 4), shared by the single solve
// (st_solve.cu) and the batched solve (st_batch.cu): workspace slots, the
// small host-side problems (rank decisions of the block QR, Ritz values,
// adaptive shifts, the projected time recurrence) and the synchronous helpers
// the rare fallback paths use.
#pragma once

#include <chrono>
#include <vector>

#include "st_common.cuh"

namespace rksm {

using Clock = std::chrono::steady_clock;
inline double ms_since(Clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
}

enum SlotId {
    S_F1D = 0, S_F1C, S_MAQ, S_WH, S_WH2, S_TMP, S_X32, S_W32, S_T32, S_SMALL, S_PART, S_COPY, S_MV,
    S_RES, S_RESP, S_LRQ, S_LRZ, S_CNF1, S_CNF2, S_CNBUF, S_CNTMP, S_GZ, S_GT, S_WDF, S_GH, S_GHD, S_GPART,
    S_CG, S_CGS
};

struct Ctx {
    st_problem* p;
    cudaStream_t s;
    int n;
};

struct HostSym {
    std::vector<double> a;
    int ld = 0;
    void grow(int need) {
        if (need <= ld) return;
        int nl = std::max(need, 2 * ld + 16);
        std::vector<double> b((size_t)nl * nl, 0.0);
        for (int j = 0; j < ld; ++j)
            for (int i = 0; i < ld; ++i) b[(size_t)j * nl + i] = a[(size_t)j * ld + i];
        a.swap(b);
        ld = nl;
    }
    double& operator()(int i, int j) { return a[(size_t)j * ld + i]; }
};

inline size_t pad32(size_t m) { return (m + 31) & ~size_t(31); }

struct QrPlan {
    int rank = 0;
    bool fast = false;
    bool severe = false;      // a kept direction lost more than 6 digits to Gram-Schmidt
    std::vector<double> R1;   // m x m upper, ld m
};

// Records why the Krylov process broke down (text of st_last_error).
int breakdown(const char* why);
int read_dev(Ctx& c, const double* d, int ld, int rows, int cols, double* h, int ldh);
int write_dev(Ctx& c, const double* h, int ldh, int rows, int cols, double* d, int ld);
// H (host, k x m) = V^T W over the n rows (synchronises).
int ts_tn_host(Ctx& c, int k, int m, const double* V, int ldv, const double* W, int ldw, double* H);
// W = beta W + alpha V H with H given on the host (k x m).
int ts_nn_host(Ctx& c, int k, int m, double alpha, const double* V, int ldv, const double* H, double beta, double* W,
               int ldw);
// Orthonormalise the m columns of W by CholQR2 with a rank-revealing fallback (see st_solve.cu).
int block_qr(Ctx& c, double* W, int ldw, int m, double ref2, double drop, std::vector<double>& R, int* r_out);
// Adaptive shift: maximiser of prod |s - s_j| / prod |s + theta_i| over [a, b] on a log grid.
double next_shift(double a, double b, const std::vector<double>& used, const std::vector<double>& ritz, int grid);
// Ritz values of the pencil (Am, Mm) (k x k, ld ld).
bool ritz_values(int k, const double* Am, const double* Mm, int ld, std::vector<double>& out);
// Time recurrence of the projected equation Mm Y D_t^T + Am Y C_t^T = Gm F2c^T.
bool projected_solve(int k, int n_t, double dt, const double* Mm, const double* Am, int ld, const double* Gm,
                     int ldg, int r, const double* F2c, std::vector<double>& Y, bool sym = true);
// Grows the basis V (and M V, the double-float copy) to need_cols, keeping keep_cols.
int ensure_basis(st_problem* p, Ctx& c, int need_cols, int keep_cols, double** MV);
// Rank of a block from its Gram matrix and the first CholQR factor.
void qr_plan(const double* G, int m, double ref2, double drop, QrPlan& q);
// R = R2 R1 for upper triangular m x m factors.
std::vector<double> upper_product(int m, const double* R2, const double* R1);
// Iterations until the next residual check.
int check_gap(const std::vector<int>& hist_it, const std::vector<double>& hist_res, int it, double res, double tol,
              double cost);
// The single-problem driver (st_solve).
// Problems given as CSR matrices (st_pcg.cu): (cm M + ca A) X = B by Jacobi-preconditioned block CG, and the
// pencil interval of (A, M) estimated once per problem.
int pcg_solve(Ctx& c, double cm, double ca, const double* B, int ldb, int ncols, double* X, int ldx, double rtol,
              int maxit, int* iters_out);
int csr_spectrum(Ctx& c);
int solve_impl(st_problem* p, const double* F1, int ldf1, const double* F2, int ldf2, int p0, st_solution* sol,
               st_stats* st);

// The lock-step batched driver (st_batch.cu): groupable problems only.
int solve_batch_impl(int count, st_problem* const* probs, const double* const* F1, const int* ldf1,
                     const double* const* F2, const int* ldf2, const int* ncols, st_solution* sols, st_stats* stats,
                     int* status, cudaStream_t s, st_batch_stats* bs, int host_threads);

}  // namespace rksm
