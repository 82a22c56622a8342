// The wave equation's space-time system on the device (paper Section 4
// "Discretized Wave problem", Section 5 Example 2):
//     M_h U Q_t^T + A_h U (D_t + D_t^T) + Q_h U M_t = F = F1 F2^T      (eq. 3terms)
// by GMRES on vec(U), right-preconditioned by the two-term operator
// P(W) = M_h W Q_t^T + Q_h W M_t, whose inverse diagonalises the pencils
// (Q_h, M_h) and (Q_t, M_t) (S^T M S = I, S^T Q S = diag(lambda)):
//     P^{-1}(V) = S_h [ (S_h^T V S_t) ./ (lambda_h_i + lambda_t_j) ] S_t^T.
// The matrices are the cubic B-spline Gram matrices of st_wave_matrices
// (banded, |i - j| <= 3).  Device work: the three-term operator as banded
// passes (time direction, then space: 42 FMAs an entry), the preconditioner as
// four dense FP64 products and a scaling, the Arnoldi step as tall-skinny
// products over the N_h N_t entries (classical Gram-Schmidt twice).  Host
// work: the two generalised eigenproblems (Cholesky of M, the symmetric
// eigenproblem of L^{-1} Q L^{-T}), the Givens rotations and the small
// triangular solve.  X_0 = 0, no restart; stop when the residual estimate
// |g_{j+1}| / ||F||_F <= tol (right preconditioning: the true residual of the
// system).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

#include "st_common.cuh"
#include "st_rksm.h"

using namespace rksm;

namespace {

constexpr int kBand = 3, kW = 2 * kBand + 1;

// band[r * 7 + (c - r + 3)] of a column-major dense n x n matrix with |r - c| <= 3
std::vector<double> to_band(int n, const std::vector<double>& A) {
    std::vector<double> b((size_t)n * kW, 0.0);
    for (int r = 0; r < n; ++r)
        for (int c = std::max(0, r - kBand); c <= std::min(n - 1, r + kBand); ++c)
            b[(size_t)r * kW + (c - r + kBand)] = A[(size_t)c * n + r];
    return b;
}

// time pass: T_q = U Q_t^T, T_s = U S_t^T, T_m = U M_t^T (U column-major nh x nt; the time matrices banded)
__global__ void k_wave_time(int nh, int nt, const double* __restrict__ U, const double* __restrict__ bq,
                            const double* __restrict__ bs, const double* __restrict__ bm, double* __restrict__ Tq,
                            double* __restrict__ Ts, double* __restrict__ Tm) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)nh * nt) return;
    const int k = (int)(idx / nh), i = (int)(idx % nh);
    double q = 0.0, s = 0.0, m = 0.0;
#pragma unroll
    for (int d = -kBand; d <= kBand; ++d) {
        const int b = k + d;
        if (b < 0 || b >= nt) continue;
        const double u = U[(size_t)b * nh + i];
        const int e = k * kW + d + kBand;   // row k of the band, column b
        q = __fma_rn(bq[e], u, q);
        s = __fma_rn(bs[e], u, s);
        m = __fma_rn(bm[e], u, m);
    }
    Tq[idx] = q;
    Ts[idx] = s;
    Tm[idx] = m;
}

// space pass: Y = M_h T_q + A_h T_s + Q_h T_m
__global__ void k_wave_space(int nh, int nt, const double* __restrict__ Tq, const double* __restrict__ Ts,
                             const double* __restrict__ Tm, const double* __restrict__ bm, const double* __restrict__ ba,
                             const double* __restrict__ bq, double* __restrict__ Y) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)nh * nt) return;
    const int k = (int)(idx / nh), i = (int)(idx % nh);
    double y = 0.0;
#pragma unroll
    for (int d = -kBand; d <= kBand; ++d) {
        const int a = i + d;
        if (a < 0 || a >= nh) continue;
        const size_t src = (size_t)k * nh + a;
        const int e = i * kW + d + kBand;
        y = __fma_rn(bm[e], Tq[src], y);
        y = __fma_rn(ba[e], Ts[src], y);
        y = __fma_rn(bq[e], Tm[src], y);
    }
    Y[idx] = y;
}

// T[i, j] /= lh[i] + lt[j]
__global__ void k_wave_scale(int nh, int nt, double* __restrict__ T, const double* __restrict__ lh,
                             const double* __restrict__ lt) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)nh * nt) return;
    const int j = (int)(idx / nh), i = (int)(idx % nh);
    T[idx] = T[idx] / (lh[i] + lt[j]);
}

// S (column-major, S^T M S = I) and lambda of the symmetric-definite pencil (Q, M): M = L L^T,
// C = L^{-1} Q L^{-T} = E diag(lambda) E^T, S = L^{-T} E.
bool pencil_eig(int n, const std::vector<double>& Q, const std::vector<double>& M, std::vector<double>& S,
                std::vector<double>& lam) {
    std::vector<double> L = M;
    if (!dense::cholesky(n, L.data(), n)) return false;
    // C = L^{-1} Q L^{-T}: X = L^{-1} Q, then C = (L^{-1} X^T)^T = L^{-1} X^T (C symmetric)
    std::vector<double> X = Q;
    dense::lower_solve(n, L.data(), n, X.data(), n, n);
    std::vector<double> Xt((size_t)n * n);
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) Xt[(size_t)i * n + j] = X[(size_t)j * n + i];
    dense::lower_solve(n, L.data(), n, Xt.data(), n, n);
    for (int j = 0; j < n; ++j)   // symmetrise the rounding
        for (int i = j + 1; i < n; ++i) {
            const double v = 0.5 * (Xt[(size_t)j * n + i] + Xt[(size_t)i * n + j]);
            Xt[(size_t)j * n + i] = Xt[(size_t)i * n + j] = v;
        }
    lam.assign(n, 0.0);
    dense::sym_eig(n, Xt.data(), n, lam.data());   // Xt <- E
    // S = L^{-T} E: back substitution with L^T, column by column
    S = Xt;
    for (int c = 0; c < n; ++c) {
        double* s = &S[(size_t)c * n];
        for (int i = n - 1; i >= 0; --i) {
            double v = s[i];
            for (int r = i + 1; r < n; ++r) v -= L[(size_t)i * n + r] * s[r];   // (L^T)[i][r] = L[r][i]
            s[i] = v / L[(size_t)i * n + i];
        }
    }
    return true;
}

std::vector<double> transpose(int n, const std::vector<double>& A) {
    std::vector<double> T((size_t)n * n);
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) T[(size_t)i * n + j] = A[(size_t)j * n + i];
    return T;
}

}  // namespace

extern "C" int st_wave_solve(int n_x, int n_t, double T, const double* F1, int ldf1, const double* F2, int ldf2,
                             int p, double tol, int maxit, double* U, int ldu, st_stats* stats, void* stream) {
    const int nh = n_x + 1, nt = n_t + 1;
    if (n_x < 4 || n_t < 4 || !(T > 0.0) || !F1 || !F2 || p < 1 || ldf1 < nh || ldf2 < nt || !(tol > 0.0) ||
        maxit < 1 || !U || ldu < nh)
        return ST_EINVAL;
    const auto t0 = Clock::now();
    if (stats) *stats = st_stats{};
    cudaStream_t s = (cudaStream_t)stream;
    // a problem handle only for its allocator and workspace slots (no operators)
    st_problem host{};
    st_problem* P = &host;
    P->stream = s;
    P->n_h = nh * nt;
    ST_CUDA_TRY(cudaGetDevice(&P->device));
    Ctx c{P, s, nh * nt};
    const size_t L = (size_t)nh * nt;
    int rc = ST_OK;
    // ---- host: matrices, bands, the two pencil eigendecompositions ----
    std::vector<double> Mh((size_t)nh * nh), Ah((size_t)nh * nh), Qh((size_t)nh * nh), Mt((size_t)nt * nt),
        Dt((size_t)nt * nt), Qt((size_t)nt * nt);
    ST_TRY(st_wave_matrices(n_x, n_t, T, Mh.data(), Ah.data(), Qh.data(), Mt.data(), Dt.data(), Qt.data()));
    std::vector<double> St((size_t)nt * nt);
    for (int j = 0; j < nt; ++j)
        for (int i = 0; i < nt; ++i) St[(size_t)j * nt + i] = Dt[(size_t)j * nt + i] + Dt[(size_t)i * nt + j];
    std::vector<double> Sh, lh, Se, lt;
    // the two pencils on two host threads (each a dense symmetric eigenproblem)
    bool ok_t = false;
    std::thread tt([&] { ok_t = pencil_eig(nt, Qt, Mt, Se, lt); });
    const bool ok_h = pencil_eig(nh, Qh, Mh, Sh, lh);
    tt.join();
    if (!ok_h || !ok_t) {
        st_note_msg("st_wave_solve: a mass matrix is not positive definite");
        return ST_EBREAKDOWN;
    }
    const double setup_ms = ms_since(t0);
    // ---- device buffers ----
    std::vector<void*> bufs;
    auto dalloc = [&](size_t doubles, double** out) -> int {
        void* ptr = nullptr;
        if (cudaMallocAsync(&ptr, sizeof(double) * std::max<size_t>(doubles, 1), s) != cudaSuccess) {
            cudaGetLastError();
            return ST_ENOMEM;
        }
        bufs.push_back(ptr);
        *out = (double*)ptr;
        return ST_OK;
    };
    auto up = [&](const std::vector<double>& h, double** d) -> int {
        ST_TRY(dalloc(h.size(), d));
        ST_CUDA_TRY(cudaMemcpyAsync(*d, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice, s));
        return ST_OK;
    };
    auto run = [&]() -> int {
        double *bMh, *bAh, *bQh, *bMt, *bSt, *bQt, *dSh, *dShT, *dSe, *dSeT, *dlh, *dlt;
        ST_TRY(up(to_band(nh, Mh), &bMh));
        ST_TRY(up(to_band(nh, Ah), &bAh));
        ST_TRY(up(to_band(nh, Qh), &bQh));
        ST_TRY(up(to_band(nt, Mt), &bMt));
        ST_TRY(up(to_band(nt, St), &bSt));
        ST_TRY(up(to_band(nt, Qt), &bQt));
        ST_TRY(up(Sh, &dSh));
        ST_TRY(up(transpose(nh, Sh), &dShT));
        ST_TRY(up(Se, &dSe));
        ST_TRY(up(transpose(nt, Se), &dSeT));
        ST_TRY(up(lh, &dlh));
        ST_TRY(up(lt, &dlt));
        double *V, *w, *z, *T1, *T2, *tq, *ts, *tm;
        ST_TRY(dalloc(L * (size_t)(maxit + 1), &V));
        ST_TRY(dalloc(L, &w));
        ST_TRY(dalloc(L, &z));
        ST_TRY(dalloc(L, &T1));
        ST_TRY(dalloc(L, &T2));
        ST_TRY(dalloc(3 * L, &tq));
        ts = tq + L;
        tm = ts + L;
        const unsigned g = (unsigned)((L + 255) / 256);
        auto precond = [&](const double* v, double* out) -> int {   // out = P^{-1}(v)
            ST_TRY(st_gemm_cm(nh, nt, nh, dShT, nh, v, nh, T1, nh, s));    // S_h^T V
            ST_TRY(st_gemm_cm(nh, nt, nt, T1, nh, dSe, nt, T2, nh, s));    // (.) S_t
            k_wave_scale<<<g, 256, 0, s>>>(nh, nt, T2, dlh, dlt);
            ST_LAUNCH_CHECK();
            ST_TRY(st_gemm_cm(nh, nt, nh, dSh, nh, T2, nh, T1, nh, s));    // S_h (.)
            ST_TRY(st_gemm_cm(nh, nt, nt, T1, nh, dSeT, nt, out, nh, s));  // (.) S_t^T
            return ST_OK;
        };
        auto op = [&](const double* u, double* out) -> int {   // out = M_h U Q_t^T + A_h U S_t^T + Q_h U M_t^T
            k_wave_time<<<g, 256, 0, s>>>(nh, nt, u, bQt, bSt, bMt, tq, ts, tm);
            ST_LAUNCH_CHECK();
            k_wave_space<<<g, 256, 0, s>>>(nh, nt, tq, ts, tm, bMh, bAh, bQh, out);
            ST_LAUNCH_CHECK();
            return ST_OK;
        };
        // F = F1 F2^T (small factors through the host)
        std::vector<double> f1((size_t)nh * p), f2t((size_t)p * nt);
        {
            std::vector<double> a((size_t)ldf1 * p), b((size_t)ldf2 * p);
            const cudaMemcpyKind k1 = st_is_device_ptr(F1) ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
            const cudaMemcpyKind k2 = st_is_device_ptr(F2) ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
            ST_CUDA_TRY(cudaMemcpyAsync(a.data(), F1, sizeof(double) * a.size(), k1, s));
            ST_CUDA_TRY(cudaMemcpyAsync(b.data(), F2, sizeof(double) * b.size(), k2, s));
            ST_CUDA_TRY(cudaStreamSynchronize(s));
            for (int q = 0; q < p; ++q) {
                std::memcpy(&f1[(size_t)q * nh], &a[(size_t)q * ldf1], sizeof(double) * nh);
                for (int l = 0; l < nt; ++l) f2t[(size_t)l * p + q] = b[(size_t)q * ldf2 + l];
            }
        }
        double *df1, *df2t;
        ST_TRY(up(f1, &df1));
        ST_TRY(up(f2t, &df2t));
        ST_TRY(st_lowrank_dense(nh, p, nt, df1, nh, df2t, p, V, nh, s));   // v_0 <- F (normalised below)
        std::vector<double> nrm(1);
        ST_TRY(ts_tn_host(c, 1, 1, V, (int)L, V, (int)L, nrm.data()));
        const double beta = std::sqrt(std::max(nrm[0], 0.0));
        if (!(beta > 0.0)) {   // F = 0: U = 0
            for (int l = 0; l < nt; ++l) ST_CUDA_TRY(cudaMemsetAsync(U + (size_t)l * ldu, 0, sizeof(double) * nh, s));
            if (stats) stats->converged = 1;
            return ST_OK;
        }
        ST_TRY(st_axpby64((int)L, 1, 1.0 / beta, V, (int)L, 0.0, V, (int)L, s));
        std::vector<double> H((size_t)(maxit + 1) * maxit, 0.0), cs(maxit), sn(maxit), gv(maxit + 1, 0.0);
        gv[0] = beta;
        int j = 0, m = 0;
        double est = 1.0;
        bool conv = false;
        for (j = 0; j < maxit; ++j) {
            const double* vj = V + (size_t)j * L;
            ST_TRY(precond(vj, z));
            ST_TRY(op(z, w));
            // classical Gram-Schmidt twice against v_0..v_j
            std::vector<double> h(j + 1), hsum(j + 1, 0.0);
            for (int pass = 0; pass < 2; ++pass) {
                ST_TRY(ts_tn_host(c, j + 1, 1, V, (int)L, w, (int)L, h.data()));
                ST_TRY(ts_nn_host(c, j + 1, 1, -1.0, V, (int)L, h.data(), 1.0, w, (int)L));
                for (int i = 0; i <= j; ++i) hsum[i] += h[i];
            }
            ST_TRY(ts_tn_host(c, 1, 1, w, (int)L, w, (int)L, nrm.data()));
            const double hn = std::sqrt(std::max(nrm[0], 0.0));
            double* col = &H[(size_t)j * (maxit + 1)];
            for (int i = 0; i <= j; ++i) col[i] = hsum[i];
            col[j + 1] = hn;
            for (int i = 0; i < j; ++i) {
                const double a = col[i], b = col[i + 1];
                col[i] = cs[i] * a + sn[i] * b;
                col[i + 1] = -sn[i] * a + cs[i] * b;
            }
            const double r = std::hypot(col[j], col[j + 1]);
            if (!(r > 0.0)) {
                st_note_msg("st_wave_solve: GMRES breakdown (singular Hessenberg column)");
                return ST_EBREAKDOWN;
            }
            cs[j] = col[j] / r;
            sn[j] = col[j + 1] / r;
            col[j] = r;
            col[j + 1] = 0.0;
            gv[j + 1] = -sn[j] * gv[j];
            gv[j] = cs[j] * gv[j];
            est = std::fabs(gv[j + 1]) / beta;
            m = j + 1;
            if (est <= tol || hn == 0.0) {
                conv = est <= tol || hn == 0.0;
                break;
            }
            ST_TRY(st_axpby64((int)L, 1, 1.0 / hn, w, (int)L, 0.0, V + (size_t)(j + 1) * L, (int)L, s));
        }
        // y = H^{-1} g (upper triangular m x m), U = P^{-1}(V y)
        std::vector<double> y(m);
        for (int i = m - 1; i >= 0; --i) {
            double v = gv[i];
            for (int k = i + 1; k < m; ++k) v -= H[(size_t)k * (maxit + 1) + i] * y[k];
            y[i] = v / H[(size_t)i * (maxit + 1) + i];
        }
        ST_TRY(ts_nn_host(c, m, 1, 1.0, V, (int)L, y.data(), 0.0, w, (int)L));
        ST_TRY(precond(w, z));
        const cudaMemcpyKind ku = st_is_device_ptr(U) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        ST_CUDA_TRY(cudaMemcpy2DAsync(U, sizeof(double) * ldu, z, sizeof(double) * nh, sizeof(double) * nh, nt, ku, s));
        ST_CUDA_TRY(cudaStreamSynchronize(s));
        if (stats) {
            stats->iterations = m;
            stats->relres = est;
            stats->converged = conv ? 1 : 0;
            stats->ms_phase[0] = setup_ms;
        }
        return conv ? ST_OK : ST_ENOTCONV;
    };
    rc = run();
    for (void* ptr : bufs) cudaFreeAsync(ptr, s);
    for (void* ptr : host.owned) cudaFreeAsync(ptr, s);   // the workspace slots of the tall-skinny products
    host.owned.clear();
    cudaStreamSynchronize(s);
    st_pinned_put(host.sm_host, host.sm_host_bytes);   // after the stream synchronisation above
    host.sm_host = nullptr;
    cudaGetLastError();
    if (stats) stats->ms_total = ms_since(t0);
    return rc;
}
