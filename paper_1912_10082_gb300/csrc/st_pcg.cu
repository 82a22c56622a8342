// Algebraic inner solver for problems given as user CSR matrices (general
// meshes, e.g. P1 on an unstructured simplex mesh): the shifted solves of the
// rational Krylov method (paper Section 4, (A + s M)^{-1} M applied to the
// newest block) and the start block's M^{-1} F1, as a block conjugate-gradient
// iteration on (c_M M + c_A A) X = B for symmetric positive definite M and A,
// preconditioned by the inverse diagonal (Jacobi).
//
// The columns of the block are independent CG processes advanced together:
// every kernel serves all columns, and every scalar of the iteration (the step
// alpha = r.z / p.q and the direction update beta = r'.z' / r.z, per column)
// stays on the device: the dot products reduce in a fixed order into device
// arrays that the next kernel reads.  The host looks at the residual norms
// every kCheck iterations only.  A column whose r.z or p.q has become exactly
// zero takes alpha = beta = 0 (it has converged to rounding).
//
// The pencil interval [lambda_min, lambda_max] of (A, M), which the adaptive
// shifts search, is estimated once per problem from these solves: power
// iteration on M^{-1} A and inverse iteration on A^{-1} M, each ending in a
// Rayleigh quotient.
#include <algorithm>
#include <cmath>
#include <vector>

#include "st_common.cuh"
#include "st_rksm.h"

namespace {

constexpr int kPcgThreads = 256;
constexpr int kPcgChunk = 2048;   // rows per dot-product block
constexpr int kCheck = 8;         // iterations between host checks of the residual norms

// inverse of the diagonal of cm M + ca A (CSR rows with sorted columns)
__global__ void k_pcg_diag(int n, const int* __restrict__ row_ptr, const int* __restrict__ col,
                           const double* __restrict__ mv, const double* __restrict__ av, double cm, double ca,
                           double* __restrict__ dinv) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double d = 0.0;
    for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
        if (col[e] == i) d = cm * mv[e] + ca * av[e];
    dinv[i] = d > 0.0 ? 1.0 / d : 1.0;
}

// X = 0, R = B, Z = D^{-1} R, P = Z
__global__ void k_pcg_init(int n, int m, const double* __restrict__ B, long long ldb, double* __restrict__ X,
                           long long ldx, double* __restrict__ R, double* __restrict__ Z, double* __restrict__ P,
                           const double* __restrict__ dinv) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * m) return;
    const int j = (int)(idx / n), i = (int)(idx % n);
    const double b = B[(size_t)j * ldb + i];
    const double z = dinv[i] * b;
    X[(size_t)j * ldx + i] = 0.0;
    R[idx] = b;
    Z[idx] = z;
    P[idx] = z;
}

// per (chunk, column): partial sums of U1.V1 and (if U2) U2.V2 over the chunk's rows, in a fixed order
__global__ void __launch_bounds__(kPcgThreads) k_pcg_dot_partial(int n, const double* __restrict__ U1,
                                                                 const double* __restrict__ V1,
                                                                 const double* __restrict__ U2,
                                                                 const double* __restrict__ V2,
                                                                 double* __restrict__ part) {
    const int chunk = blockIdx.x, j = blockIdx.y, nch = gridDim.x;
    const int r0 = chunk * kPcgChunk, r1 = min(n, r0 + kPcgChunk);
    const size_t off = (size_t)j * n;
    double s1 = 0.0, s2 = 0.0;
    for (int i = r0 + threadIdx.x; i < r1; i += kPcgThreads) {
        s1 += U1[off + i] * V1[off + i];
        if (U2) s2 += U2[off + i] * V2[off + i];
    }
    __shared__ double sh1[kPcgThreads / 32], sh2[kPcgThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (lane == 0) {
        sh1[warp] = s1;
        sh2[warp] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t1 = 0.0, t2 = 0.0;
        for (int w = 0; w < kPcgThreads / 32; ++w) {
            t1 += sh1[w];
            t2 += sh2[w];
        }
        part[(size_t)j * nch + chunk] = t1;
        part[(size_t)(gridDim.y + j) * nch + chunk] = t2;
    }
}

// out[j] (and out[m + j]) = the chunk partials of column j summed in chunk order, one warp a value
__global__ void k_pcg_dot_reduce(int nch, int nvals, const double* __restrict__ part, double* __restrict__ out) {
    const int v = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x % 32;
    if (v >= nvals) return;
    double s = 0.0;
    for (int c = lane; c < nch; c += 32) s += part[(size_t)v * nch + c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[v] = s;
}

// alpha = rz / pq per column; X += alpha P, R -= alpha Q, Z = D^{-1} R
__global__ void k_pcg_update(int n, int m, double* __restrict__ X, long long ldx, const double* __restrict__ P,
                             double* __restrict__ R, const double* __restrict__ Q, double* __restrict__ Z,
                             const double* __restrict__ dinv, const double* __restrict__ rz,
                             const double* __restrict__ pq) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * m) return;
    const int j = (int)(idx / n), i = (int)(idx % n);
    const double den = pq[j];
    const double alpha = den != 0.0 ? rz[j] / den : 0.0;
    X[(size_t)j * ldx + i] = __fma_rn(alpha, P[idx], X[(size_t)j * ldx + i]);
    const double r = __fma_rn(-alpha, Q[idx], R[idx]);
    R[idx] = r;
    Z[idx] = dinv[i] * r;
}

// beta = rz_new / rz_old per column; P = Z + beta P
__global__ void k_pcg_direction(int n, int m, double* __restrict__ P, const double* __restrict__ Z,
                                const double* __restrict__ rz_new, const double* __restrict__ rz_old) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * m) return;
    const int j = (int)(idx / n);
    const double den = rz_old[j];
    const double beta = den != 0.0 ? rz_new[j] / den : 0.0;
    P[idx] = __fma_rn(beta, P[idx], Z[idx]);
}

inline unsigned grid_of(long long total) { return (unsigned)((total + kPcgThreads - 1) / kPcgThreads); }

}  // namespace

namespace rksm {

// (cm M + ca A) X = B for ncols <= 16 columns by Jacobi-preconditioned CG; stops when every column's residual
// is at most rtol times its right-hand side's norm (ST_ENOTCONV after maxit iterations, X the last iterate).
int pcg_solve(Ctx& c, double cm, double ca, const double* B, int ldb, int ncols, double* X, int ldx, double rtol,
              int maxit, int* iters_out) {
    st_problem* p = c.p;
    const int n = c.n, m = ncols;
    if (iters_out) *iters_out = 0;
    if (n <= 0 || m <= 0) return ST_OK;
    if (m > 16) return ST_EINVAL;
    const size_t nm = (size_t)n * m;
    const int nch = (n + kPcgChunk - 1) / kPcgChunk;
    double *vecs, *small;
    ST_TRY(st_slot(p, S_CG, sizeof(double) * 4 * nm, (void**)&vecs));
    // small: dinv (n) | partials (2 m nch) | dots: rz, rz', pq, rr, bb (m each; rr and bb adjacent)
    ST_TRY(st_slot(p, S_CGS, sizeof(double) * ((size_t)n + 2 * (size_t)m * nch + 6 * (size_t)m), (void**)&small));
    double *R = vecs, *Z = vecs + nm, *P = vecs + 2 * nm, *Q = vecs + 3 * nm;
    double* dinv = small;
    double* part = small + n;
    double* dots = part + 2 * (size_t)m * nch;
    double *rz = dots, *rz2 = dots + m, *pq = dots + 2 * m, *rr = dots + 3 * m, *bb = dots + 4 * m;
    const dim3 dgrid(nch, m);
    auto dot2 = [&](const double* u1, const double* v1, const double* u2, const double* v2, double* out1) -> int {
        k_pcg_dot_partial<<<dgrid, kPcgThreads, 0, c.s>>>(n, u1, v1, u2, v2, part);
        ST_LAUNCH_CHECK();
        // out1[0..m) from the first products; the second products land right after (out1 + m)
        k_pcg_dot_reduce<<<(2 * m + 7) / 8, 256, 0, c.s>>>(nch, u2 ? 2 * m : m, part, out1);
        ST_LAUNCH_CHECK();
        return ST_OK;
    };
    k_pcg_diag<<<grid_of(n), kPcgThreads, 0, c.s>>>(n, p->row_ptr, p->col, p->m64, p->a64, cm, ca, dinv);
    ST_LAUNCH_CHECK();
    k_pcg_init<<<grid_of((long long)nm), kPcgThreads, 0, c.s>>>(n, m, B, ldb, X, ldx, R, Z, P, dinv);
    ST_LAUNCH_CHECK();
    ST_TRY(dot2(R, R, nullptr, nullptr, rr));
    ST_CUDA_TRY(cudaMemcpyAsync(bb, rr, sizeof(double) * m, cudaMemcpyDeviceToDevice, c.s));
    ST_TRY(dot2(R, Z, nullptr, nullptr, rz));
    std::vector<double> hb(m), hr(m);
    ST_CUDA_TRY(cudaMemcpyAsync(hb.data(), bb, sizeof(double) * m, cudaMemcpyDeviceToHost, c.s));
    ST_CUDA_TRY(cudaStreamSynchronize(c.s));
    bool done = true;
    for (int j = 0; j < m; ++j) done = done && hb[j] == 0.0;
    if (done) return ST_OK;   // B = 0: X = 0
    const double tol2 = rtol * rtol;
    int it = 0;
    while (it < maxit) {
        ++it;
        ST_TRY(st_spmm_comb64(p, cm, ca, P, n, m, 0.0, Q, n, c.s));   // Q = (cm M + ca A) P
        ST_TRY(dot2(P, Q, nullptr, nullptr, pq));
        k_pcg_update<<<grid_of((long long)nm), kPcgThreads, 0, c.s>>>(n, m, X, ldx, P, R, Q, Z, dinv, rz, pq);
        ST_LAUNCH_CHECK();
        // rz' = r.z and rr = r.r (rz2 and rr are not adjacent: two reductions into their own arrays)
        ST_TRY(dot2(R, Z, nullptr, nullptr, rz2));
        k_pcg_direction<<<grid_of((long long)nm), kPcgThreads, 0, c.s>>>(n, m, P, Z, rz2, rz);
        ST_LAUNCH_CHECK();
        std::swap(rz, rz2);
        if (it % kCheck == 0 || it == maxit) {
            ST_TRY(dot2(R, R, nullptr, nullptr, rr));
            ST_CUDA_TRY(cudaMemcpyAsync(hr.data(), rr, sizeof(double) * m, cudaMemcpyDeviceToHost, c.s));
            ST_CUDA_TRY(cudaStreamSynchronize(c.s));
            done = true;
            for (int j = 0; j < m; ++j) done = done && hr[j] <= tol2 * hb[j];
            if (done) break;
        }
    }
    if (iters_out) *iters_out = it;
    return done ? ST_OK : ST_ENOTCONV;
}

// lambda_min and lambda_max of the pencil (A, M) for a problem given as CSR matrices (once per problem):
// 30 power steps on M^{-1} A and 12 inverse steps on A^{-1} M from a seeded start, each a Rayleigh
// quotient x^T A x / x^T M x at the end.  The adaptive shifts only need the interval roughly.
int csr_spectrum(Ctx& c) {
    st_problem* p = c.p;
    if (p->lam_max > 0.0) return ST_OK;
    const int n = c.n;
    double *x, *y;
    ST_TRY(st_slot(p, S_TMP, sizeof(double) * 2 * (size_t)n, (void**)&x));
    y = x + n;
    std::vector<double> h(n);
    for (int i = 0; i < n; ++i) {
        uint32_t v = (uint32_t)i * 2654435761u + 0x9e3779b9u;
        v ^= v >> 15;
        v *= 0x85ebca6bu;
        v ^= v >> 13;
        h[i] = 0.5 + (double)(v >> 8) / 16777216.0;   // positive: overlaps the smoothest mode
    }
    auto rayleigh = [&](double* v, double* out) -> int {
        std::vector<double> xa(2);
        double* MA;
        ST_TRY(st_slot(p, S_GT, sizeof(double) * 2 * (size_t)n, (void**)&MA));
        ST_TRY(st_spmm_ma<double>(p, v, n, 1, MA, n, MA + n, n, c.s));
        std::vector<double> g(2);
        ST_TRY(ts_tn_host(c, 1, 2, v, n, MA, n, g.data()));   // [x^T M x, x^T A x]
        *out = g[0] > 0.0 ? g[1] / g[0] : 0.0;
        return ST_OK;
    };
    auto normalise = [&](double* v) -> int {
        std::vector<double> g(1);
        ST_TRY(ts_tn_host(c, 1, 1, v, n, v, n, g.data()));
        const double s = g[0] > 0.0 ? 1.0 / std::sqrt(g[0]) : 1.0;
        return st_axpby64(n, 1, s, v, n, 0.0, v, n, c.s);
    };
    double lmax = 0.0, lmin = 0.0;
    ST_CUDA_TRY(cudaMemcpyAsync(x, h.data(), sizeof(double) * n, cudaMemcpyHostToDevice, c.s));
    for (int it = 0; it < 30; ++it) {   // x <- M^{-1} A x
        ST_TRY(st_spmm_comb64(p, 0.0, 1.0, x, n, 1, 0.0, y, n, c.s));
        int its = 0;
        const int rc = pcg_solve(c, 1.0, 0.0, y, n, 1, x, n, 1e-8, 2000, &its);
        if (rc != ST_OK && rc != ST_ENOTCONV) return rc;
        ST_TRY(normalise(x));
    }
    ST_TRY(rayleigh(x, &lmax));
    ST_CUDA_TRY(cudaMemcpyAsync(x, h.data(), sizeof(double) * n, cudaMemcpyHostToDevice, c.s));
    for (int it = 0; it < 12; ++it) {   // x <- A^{-1} M x
        ST_TRY(st_spmm_comb64(p, 1.0, 0.0, x, n, 1, 0.0, y, n, c.s));
        int its = 0;
        const int rc = pcg_solve(c, 0.0, 1.0, y, n, 1, x, n, 1e-8, 20000, &its);
        if (rc != ST_OK && rc != ST_ENOTCONV) return rc;
        ST_TRY(normalise(x));
    }
    ST_TRY(rayleigh(x, &lmin));
    if (!(lmax > 0.0) || !(lmin > 0.0)) return breakdown("CSR problem: pencil (A, M) not positive definite");
    // the power iteration approaches lambda_max from below and the inverse iteration lambda_min from above
    p->lam_max = 1.05 * lmax;
    p->lam_min = 0.95 * lmin;
    return ST_OK;
}

}  // namespace rksm
