// Problem set-up: spatial matrices on the device, fast-diagonalisation tables,
// manufactured loads, handle bookkeeping (paper Section 3).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <climits>
#include <map>
#include <mutex>
#include <string>

#include "st_common.cuh"

static thread_local char g_last_error[512] = "";

void st_note_cuda(cudaError_t e, const char* what, const char* file, int line) {
    std::snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
}

void st_note_msg(const char* msg) { std::snprintf(g_last_error, sizeof(g_last_error), "%s", msg); }

extern "C" const char* st_last_error(void) { return g_last_error; }

extern "C" const char* st_error_string(int status) {
    switch (status) {
        case ST_OK: return "ok";
        case ST_EINVAL: return "invalid argument";
        case ST_ENOMEM: return "out of memory";
        case ST_ENOTCONV: return "not converged to the requested tolerance";
        case ST_EBREAKDOWN: return "Krylov breakdown with nothing left to add";
        case ST_ECUDA: return "CUDA error";
        case ST_ETIMEOUT: return "device wait timed out";
        case ST_ENOTSUP: return "operation not supported for this problem";
        default: return "unknown status";
    }
}

// Device memory of a handle comes from the device's stream-ordered pool
// (cudaMallocAsync / cudaFreeAsync on the handle's stream): growing or
// releasing a buffer never synchronises the device, so handles that run
// concurrently on other streams (the executor's slots) are not stalled.  The
// pool keeps freed memory for reuse instead of returning it to the driver.
static void keep_pool_memory() {
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return;
    }
    std::lock_guard<std::mutex> lk(mu);
    if (done[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        unsigned long long keep = ~0ULL;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
    done[dev] = true;
}

namespace {
std::mutex g_pin_mu;
std::multimap<size_t, void*> g_pin_free;   // pooled pinned buffers by size (powers of two from 64 KiB)
}  // namespace

void* st_pinned_get(size_t bytes, size_t* got) {
    size_t c = (size_t)64 << 10;
    while (c < bytes) c <<= 1;
    {
        std::lock_guard<std::mutex> lk(g_pin_mu);
        auto it = g_pin_free.lower_bound(c);
        if (it != g_pin_free.end() && it->first <= 4 * c) {   // a pooled buffer at most 4x the class
            void* ptr = it->second;
            *got = it->first;
            g_pin_free.erase(it);
            return ptr;
        }
    }
    void* ptr = nullptr;
    if (cudaMallocHost(&ptr, c) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    *got = c;
    return ptr;
}

void st_pinned_put(void* ptr, size_t bytes) {
    if (!ptr) return;
    std::lock_guard<std::mutex> lk(g_pin_mu);
    g_pin_free.emplace(bytes, ptr);
}

int st_alloc(st_problem* p, void** ptr, size_t bytes) {
    *ptr = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMallocAsync(ptr, bytes, p->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        st_note_cuda(e, "cudaMallocAsync", __FILE__, __LINE__);
        *ptr = nullptr;
        return e == cudaErrorMemoryAllocation ? ST_ENOMEM : ST_ECUDA;
    }
    p->owned.push_back(*ptr);
    return ST_OK;
}

int st_free_one(st_problem* p, void* ptr) {
    if (!ptr) return ST_OK;
    for (size_t i = 0; i < p->owned.size(); ++i) {
        if (p->owned[i] == ptr) {
            p->owned[i] = p->owned.back();
            p->owned.pop_back();
            break;
        }
    }
    cudaFreeAsync(ptr, p->stream);
    return ST_OK;
}

bool st_is_device_ptr(const void* ptr) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int st_stage_matrix(st_problem* p, const double* src, int ld, int rows, int cols, double* dst) {
    if (rows == 0 || cols == 0) return ST_OK;
    cudaMemcpyKind kind = st_is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    ST_CUDA_TRY(cudaMemcpy2DAsync(dst, sizeof(double) * rows, src, sizeof(double) * ld,
                                  sizeof(double) * rows, cols, kind, p->stream));
    return ST_OK;
}

// ---------------------------------------------------------------------------
// Q1 assembly.  Entry (i, j) of a Kronecker product of 1D tridiagonal factors
// depends only on the per-direction offsets d = j - i in {-1, 0, 1}.  The
// factors are multiplied slowest direction first, and the stiffness terms are
// summed x, y, z, so every value is a fixed sequence of correctly rounded
// operations (no fused multiply-add).
// ---------------------------------------------------------------------------
struct Axis1D {
    double m0, m1;   // mass diagonal 4h/6, off-diagonal h/6
    double k0, k1;   // stiffness diagonal 2/h, off-diagonal -1/h
};

__device__ __forceinline__ int prefix_1d(int i, int n) { return 3 * i - (i >= 1) - (i >= n); }
__device__ __forceinline__ int count_1d(int i, int n) { return 3 - (i == 0) - (i == n - 1); }

__device__ __forceinline__ double mval(const Axis1D& a, int d) { return d == 0 ? a.m0 : a.m1; }
__device__ __forceinline__ double kval(const Axis1D& a, int d) { return d == 0 ? a.k0 : a.k1; }
__device__ __forceinline__ double gval(int d) { return d == 0 ? 0.0 : 0.5 * d; }

__global__ void k_assemble_tensor(int dim, int nx, int ny, int nz, Axis1D ax, Axis1D ay, Axis1D az,
                                  int op, double kappa, double eps, double bx, double by, double bz,
                                  double half_dt, int n_h, int nnz, int* __restrict__ row_ptr,
                                  int* __restrict__ col, double* __restrict__ m64, double* __restrict__ a64, double* __restrict__ at64,
                                  double* __restrict__ p64, double* __restrict__ q64,
                                  float* __restrict__ m32, float* __restrict__ a32, float* __restrict__ p32,
                                  float* __restrict__ q32) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_h) return;
    int ix = r % nx;
    int t = r / nx;
    int iy = t % ny;
    int iz = t / ny;
    int cx = prefix_1d(nx, nx), cy = prefix_1d(ny, ny);
    int e = cx * cy * prefix_1d(iz, nz) + cx * count_1d(iz, nz) * prefix_1d(iy, ny) +
            count_1d(iy, ny) * count_1d(iz, nz) * prefix_1d(ix, nx);
    row_ptr[r] = e;
    if (r == n_h - 1) row_ptr[n_h] = nnz;
    int zlo = dim >= 3 ? -1 : 0, zhi = dim >= 3 ? 1 : 0;
    int ylo = dim >= 2 ? -1 : 0, yhi = dim >= 2 ? 1 : 0;
    for (int dz = zlo; dz <= zhi; ++dz) {
        int jz = iz + dz;
        if (jz < 0 || jz >= nz) continue;
        for (int dy = ylo; dy <= yhi; ++dy) {
            int jy = iy + dy;
            if (jy < 0 || jy >= ny) continue;
            for (int dx = -1; dx <= 1; ++dx) {
                int jx = ix + dx;
                if (jx < 0 || jx >= nx) continue;
                double mx = mval(ax, dx), kx = kval(ax, dx), gx = gval(dx);
                double mv, stiff, conv;
                if (dim == 1) {
                    mv = mx;
                    stiff = kx;
                    conv = __dmul_rn(bx, gx);
                } else if (dim == 2) {
                    double my = mval(ay, dy), ky = kval(ay, dy), gy = gval(dy);
                    mv = __dmul_rn(my, mx);
                    stiff = __dadd_rn(__dmul_rn(my, kx), __dmul_rn(ky, mx));
                    conv = __dadd_rn(__dmul_rn(bx, __dmul_rn(my, gx)), __dmul_rn(by, __dmul_rn(gy, mx)));
                } else {
                    // left-associated Kronecker chain ((z (x) y) (x) x)
                    double my = mval(ay, dy), ky = kval(ay, dy), gy = gval(dy);
                    double mz = mval(az, dz), kz = kval(az, dz), gz = gval(dz);
                    double mzy = __dmul_rn(mz, my);
                    mv = __dmul_rn(mzy, mx);
                    double tx = __dmul_rn(mzy, kx);
                    double ty = __dmul_rn(__dmul_rn(mz, ky), mx);
                    double tz = __dmul_rn(__dmul_rn(kz, my), mx);
                    stiff = __dadd_rn(__dadd_rn(tx, ty), tz);
                    double cxv = __dmul_rn(bx, __dmul_rn(mzy, gx));
                    double cyv = __dmul_rn(by, __dmul_rn(__dmul_rn(mz, gy), mx));
                    double czv = __dmul_rn(bz, __dmul_rn(__dmul_rn(gz, my), mx));
                    conv = __dadd_rn(__dadd_rn(cxv, cyv), czv);
                }
                double av = op == ST_CONVDIFF ? __dadd_rn(__dmul_rn(eps, stiff), conv) : __dmul_rn(kappa, stiff);
                // A^T on the same pattern: the stiffness and mass factors are
                // symmetric in the offsets, the convection factor G is skew
                double atv = op == ST_CONVDIFF ? __dsub_rn(__dmul_rn(eps, stiff), conv) : av;
                double pv = __dadd_rn(mv, __dmul_rn(half_dt, av));
                double qv = __dsub_rn(mv, __dmul_rn(half_dt, av));
                col[e] = (jz * ny + jy) * nx + jx;
                m64[e] = mv;
                a64[e] = av;
                at64[e] = atv;
                p64[e] = pv;
                q64[e] = qv;
                m32[e] = (float)mv;
                a32[e] = (float)av;
                p32[e] = (float)pv;
                q32[e] = (float)qv;
                ++e;
            }
        }
    }
}

// Fast-diagonalisation tables of one direction: the sine modes
// s_j(x_i) = sin(j i pi/(n+1)) are eigenvectors of both 1D matrices,
// M s_j = mu_j s_j with mu_j = h (4 + 2 cos(j pi/(n+1)))/6 and
// K s_j = lam_j M s_j with lam_j = (6/h^2)(1 - cos)/(2 + cos).
__global__ void k_fd_tables(int n, double h, double* __restrict__ Q64, float* __restrict__ Q32,
                            double* __restrict__ lam, double* __restrict__ c2, float* __restrict__ lam32,
                            float* __restrict__ c232) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < n * n) {
        int j = idx / n, i = idx % n;
        long long m = (long long)(j + 1) * (i + 1) % (2LL * (n + 1));
        double v = sinpi((double)m / (double)(n + 1));
        Q64[idx] = v;
        Q32[idx] = (float)v;
    }
    if (idx < n) {
        int j = idx + 1;
        double s = sinpi((double)j / (2.0 * (n + 1)));
        double c = cospi((double)j / (double)(n + 1));
        lam[idx] = (6.0 / (h * h)) * (2.0 * s * s) / (2.0 + c);
        double mu = h * (4.0 + 2.0 * c) / 6.0;
        c2[idx] = 2.0 / ((n + 1) * mu);
        lam32[idx] = (float)lam[idx];
        c232[idx] = (float)c2[idx];
    }
}

// Folded half tables of the sine matrix for the mode products (see k_gemm_fold).
__global__ void k_fd_fold_tables(int n, const double* __restrict__ Q, double* __restrict__ H0, double* __restrict__ H1,
                                 double* __restrict__ G0, double* __restrict__ G1, float* __restrict__ h0,
                                 float* __restrict__ h1, float* __restrict__ g0, float* __restrict__ g1) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int K0 = (n + 1) / 2, K1 = n / 2;
    if (idx < K0 * K0) {
        int k = idx / K0, i = idx % K0;
        double v = Q[(size_t)k * n + 2 * i];
        H0[(size_t)k * K0 + i] = v;
        G0[(size_t)i * K0 + k] = v;
        h0[(size_t)k * K0 + i] = (float)v;
        g0[(size_t)i * K0 + k] = (float)v;
    }
    if (idx < K1 * K1) {
        int k = idx / K1, i = idx % K1;
        double v = Q[(size_t)k * n + 2 * i + 1];
        H1[(size_t)k * K1 + i] = v;
        G1[(size_t)i * K1 + k] = v;
        h1[(size_t)k * K1 + i] = (float)v;
        g1[(size_t)i * K1 + k] = (float)v;
    }
}

__global__ void k_csr_copy_f32(int nnz, const double* __restrict__ m, const double* __restrict__ a, double half_dt,
                               double* __restrict__ p64, double* __restrict__ q64, float* __restrict__ m32,
                               float* __restrict__ a32, float* __restrict__ p32, float* __restrict__ q32) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    double mv = m[e], av = a[e];
    double pv = __dadd_rn(mv, __dmul_rn(half_dt, av));
    double qv = __dsub_rn(mv, __dmul_rn(half_dt, av));
    p64[e] = pv;
    q64[e] = qv;
    m32[e] = (float)mv;
    a32[e] = (float)av;
    p32[e] = (float)pv;
    q32[e] = (float)qv;
}

static int alloc_csr(st_problem* p) {
    size_t nnz = (size_t)p->nnz;
    ST_TRY(st_alloc(p, (void**)&p->row_ptr, sizeof(int) * (p->n_h + 1)));
    ST_TRY(st_alloc(p, (void**)&p->col, sizeof(int) * nnz));
    ST_TRY(st_alloc(p, (void**)&p->at64, sizeof(double) * nnz));
    double** d64[4] = {&p->m64, &p->a64, &p->p64, &p->q64};
    float** d32[4] = {&p->m32, &p->a32, &p->p32, &p->q32};
    for (int i = 0; i < 4; ++i) ST_TRY(st_alloc(p, (void**)d64[i], sizeof(double) * nnz));
    for (int i = 0; i < 4; ++i) ST_TRY(st_alloc(p, (void**)d32[i], sizeof(float) * nnz));
    return ST_OK;
}

// Values of M, A, P, N for the problem's current operator and coefficients
// (pattern and values are written together by one kernel).
static int assemble_tensor(st_problem* p) {
    const st_desc& d = p->d;
    Axis1D a1[3];
    for (int i = 0; i < 3; ++i) {
        double h = p->len[i] / (p->n[i] + 1);
        a1[i].m0 = 4.0 * h / 6.0;
        a1[i].m1 = h / 6.0;
        a1[i].k0 = 2.0 / h;
        a1[i].k1 = -1.0 / h;
    }
    int threads = 256;
    int blocks = (p->n_h + threads - 1) / threads;
    k_assemble_tensor<<<blocks, threads, 0, p->stream>>>(
        d.dim, p->n[0], p->n[1], p->n[2], a1[0], a1[1], a1[2], d.op, p->kappa, d.eps, d.beta[0], d.beta[1],
        d.beta[2], 0.5 * p->dt, p->n_h, p->nnz, p->row_ptr, p->col, p->m64, p->a64, p->at64, p->p64, p->q64, p->m32,
        p->a32, p->p32, p->q32);
    ST_LAUNCH_CHECK();
    return ST_OK;
}

// Stencil of P and N for the box-grid apply: the values of an interior row, in
// CSR (= (dz, dy, dx) lexicographic) order, placed at 27-point indices.
static int read_box_stencil(st_problem* p) {
    p->box_ok = false;
    if (p->dim < 2) return ST_OK;
    for (int d = 0; d < p->dim; ++d)
        if (p->n[d] < 3) return ST_OK;
    const int nx = p->n[0], ny = p->n[1];
    const int r = p->dim == 2 ? 1 + nx : 1 + nx * (1 + ny);
    int rp[2];
    ST_CUDA_TRY(cudaMemcpyAsync(rp, p->row_ptr + r, sizeof(int) * 2, cudaMemcpyDeviceToHost, p->stream));
    ST_CUDA_TRY(cudaStreamSynchronize(p->stream));
    const int cnt = rp[1] - rp[0];
    const int want = p->dim == 2 ? 9 : 27;
    if (cnt != want) return ST_OK;
    double v64[4][27];
    float v32[4][27];
    const double* s64[4] = {p->p64, p->q64, p->m64, p->a64};
    const float* s32[4] = {p->p32, p->q32, p->m32, p->a32};
    for (int j = 0; j < 4; ++j) {
        ST_CUDA_TRY(cudaMemcpyAsync(v64[j], s64[j] + rp[0], sizeof(double) * cnt, cudaMemcpyDeviceToHost, p->stream));
        ST_CUDA_TRY(cudaMemcpyAsync(v32[j], s32[j] + rp[0], sizeof(float) * cnt, cudaMemcpyDeviceToHost, p->stream));
    }
    ST_CUDA_TRY(cudaStreamSynchronize(p->stream));
    const int base = p->dim == 2 ? 9 : 0;   // 2D: the dz = 0 plane
    double* d64[4] = {p->box_p64, p->box_q64, p->box_m64, p->box_a64};
    float* d32[4] = {p->box_p32, p->box_q32, p->box_m32, p->box_a32};
    for (int j = 0; j < 4; ++j)
        for (int e = 0; e < 27; ++e) {
            d64[j][e] = e >= base && e < base + cnt ? v64[j][e - base] : 0.0;
            d32[j][e] = e >= base && e < base + cnt ? v32[j][e - base] : 0.f;
        }
    p->box_ok = true;
    return ST_OK;
}

// Spectrum bounds of the pencil (A, M) (heat) or of its symmetric diffusion
// part (convection-diffusion), from the 1D sine-mode eigenvalues.
static void set_spectrum(st_problem* p) {
    p->tensor_heat = p->d.op == ST_HEAT;
    p->fd_kappa = p->d.op == ST_HEAT ? p->kappa : p->d.eps;
    p->lam_min = p->fd_kappa * p->fd_lam_min;
    p->lam_max = p->fd_kappa * p->fd_lam_max;
}

static int setup_tensor(st_problem* p) {
    const st_desc& d = p->d;
    p->dim = d.dim;
    long long nh = 1;
    for (int i = 0; i < 3; ++i) {
        p->n[i] = i < d.dim ? d.n[i] : 1;
        p->len[i] = (i < d.dim && d.length[i] > 0) ? d.length[i] : 1.0;
        if (p->n[i] < 1) return ST_EINVAL;
        nh *= p->n[i];
    }
    long long nnz = 1;
    for (int i = 0; i < 3; ++i) nnz *= (i < d.dim) ? (3LL * p->n[i] - 2) : 1LL;
    if (nh > INT_MAX || nnz > INT_MAX) return ST_EINVAL;
    p->n_h = (int)nh;
    p->nnz = (int)nnz;
    p->max_row_nnz = d.dim == 1 ? 3 : (d.dim == 2 ? 9 : 27);
    ST_TRY(alloc_csr(p));
    ST_TRY(assemble_tensor(p));
    {
        p->fd_lam_min = 0.0;
        p->fd_lam_max = 0.0;
        for (int i = 0; i < d.dim; ++i) {
            FdAxis& ax = p->ax[i];
            ax.n = p->n[i];
            ax.h = p->len[i] / (ax.n + 1);
            size_t nn = (size_t)ax.n * ax.n;
            ST_TRY(st_alloc(p, (void**)&ax.Q64, sizeof(double) * nn));
            ST_TRY(st_alloc(p, (void**)&ax.Q32, sizeof(float) * nn));
            ST_TRY(st_alloc(p, (void**)&ax.lam, sizeof(double) * ax.n));
            ST_TRY(st_alloc(p, (void**)&ax.c2, sizeof(double) * ax.n));
            ST_TRY(st_alloc(p, (void**)&ax.lam32, sizeof(float) * ax.n));
            ST_TRY(st_alloc(p, (void**)&ax.c232, sizeof(float) * ax.n));
            int nb = (int)((nn + 255) / 256);
            k_fd_tables<<<nb, 256, 0, p->stream>>>(ax.n, ax.h, ax.Q64, ax.Q32, ax.lam, ax.c2, ax.lam32, ax.c232);
            ST_LAUNCH_CHECK();
            {
                const size_t k0 = (size_t)(ax.n + 1) / 2, k1 = (size_t)ax.n / 2;
                for (int t = 0; t < 4; ++t) {
                    size_t cnt = t % 2 == 0 ? k0 * k0 : k1 * k1;
                    ST_TRY(st_alloc(p, (void**)&ax.fold64[t], sizeof(double) * (cnt ? cnt : 1)));
                    ST_TRY(st_alloc(p, (void**)&ax.fold32[t], sizeof(float) * (cnt ? cnt : 1)));
                }
                int nbf = (int)((k0 * k0 + 255) / 256);
                k_fd_fold_tables<<<nbf, 256, 0, p->stream>>>(ax.n, ax.Q64, ax.fold64[0], ax.fold64[1], ax.fold64[2],
                                                             ax.fold64[3], ax.fold32[0], ax.fold32[1], ax.fold32[2],
                                                             ax.fold32[3]);
                ST_LAUNCH_CHECK();
            }
            double h = ax.h;
            auto lamj = [&](int j) {
                double s = std::sin(M_PI * j / (2.0 * (ax.n + 1)));
                double c = std::cos(M_PI * j / (ax.n + 1.0));
                return (6.0 / (h * h)) * (2.0 * s * s) / (2.0 + c);
            };
            p->fd_lam_min += lamj(1);
            p->fd_lam_max += lamj(ax.n);
        }
    }
    set_spectrum(p);
    return read_box_stencil(p);
}

static int setup_user_csr(st_problem* p, const st_desc& d) {
    if (d.n_h < 1 || d.nnz < 1 || !d.row_ptr || !d.col_idx || !d.m_vals || !d.a_vals) return ST_EINVAL;
    if (d.row_ptr[0] != 0 || d.row_ptr[d.n_h] != d.nnz) return ST_EINVAL;
    int maxr = 0;
    for (int i = 0; i < d.n_h; ++i) {
        int a = d.row_ptr[i], b = d.row_ptr[i + 1];
        if (b < a) return ST_EINVAL;
        maxr = b - a > maxr ? b - a : maxr;
        for (int e = a; e < b; ++e) {
            int c = d.col_idx[e];
            if (c < 0 || c >= d.n_h) return ST_EINVAL;
            if (e > a && c <= d.col_idx[e - 1]) return ST_EINVAL;
        }
    }
    p->dim = 0;
    p->n_h = d.n_h;
    p->nnz = d.nnz;
    p->max_row_nnz = maxr;
    ST_TRY(alloc_csr(p));
    ST_CUDA_TRY(cudaMemcpyAsync(p->row_ptr, d.row_ptr, sizeof(int) * (p->n_h + 1), cudaMemcpyHostToDevice, p->stream));
    ST_CUDA_TRY(cudaMemcpyAsync(p->col, d.col_idx, sizeof(int) * p->nnz, cudaMemcpyHostToDevice, p->stream));
    ST_CUDA_TRY(cudaMemcpyAsync(p->m64, d.m_vals, sizeof(double) * p->nnz, cudaMemcpyHostToDevice, p->stream));
    ST_CUDA_TRY(cudaMemcpyAsync(p->a64, d.a_vals, sizeof(double) * p->nnz, cudaMemcpyHostToDevice, p->stream));
    int blocks = (p->nnz + 255) / 256;
    k_csr_copy_f32<<<blocks, 256, 0, p->stream>>>(p->nnz, p->m64, p->a64, 0.5 * p->dt, p->p64, p->q64, p->m32,
                                                  p->a32, p->p32, p->q32);
    ST_LAUNCH_CHECK();
    return ST_OK;
}

extern "C" int st_destroy(st_problem* p) {
    if (!p) return ST_OK;
    if (p->cn_graph) cudaGraphExecDestroy((cudaGraphExec_t)p->cn_graph);
    for (void* ptr : p->owned) cudaFreeAsync(ptr, p->stream);
    cudaStreamSynchronize(p->stream);
    st_pinned_put(p->sm_host, p->sm_host_bytes);   // no copy in flight uses it now
    cudaGetLastError();
    p->owned.clear();
    delete p;
    return ST_OK;
}

extern "C" int st_set_coefficients(st_problem* p, int op, double kappa, double eps, const double* beta) {
    if (!p) return ST_EINVAL;
    if (p->dim < 1) return ST_ENOTSUP;
    if (op != ST_HEAT && op != ST_CONVDIFF) return ST_EINVAL;
    if (op == ST_CONVDIFF && !(eps > 0)) return ST_EINVAL;
    if (kappa < 0) return ST_EINVAL;
    double kap = kappa > 0 ? kappa : 1.0;
    bool same = op == p->d.op && kap == p->kappa && (op == ST_HEAT || eps == p->d.eps);
    for (int i = 0; i < 3 && same && op == ST_CONVDIFF; ++i) same = (beta ? beta[i] : 0.0) == p->d.beta[i];
    if (same) return ST_OK;
    p->d.op = op;
    p->kappa = kap;
    p->d.kappa = kap;
    p->d.eps = eps;
    for (int i = 0; i < 3; ++i) p->d.beta[i] = beta ? beta[i] : 0.0;
    // the captured Crank-Nicolson graph and the line factors hold the old coefficients
    p->cn_stale = true;
    p->line_valid = false;
    ST_TRY(assemble_tensor(p));
    set_spectrum(p);
    return read_box_stencil(p);
}

extern "C" int st_setup(const st_desc* d, st_problem** out) {
    if (!out) return ST_EINVAL;
    *out = nullptr;
    if (!d) return ST_EINVAL;
    if (d->dim < 0 || d->dim > 3 || d->n_t < 1 || !(d->T > 0)) return ST_EINVAL;
    if (d->op != ST_HEAT && d->op != ST_CONVDIFF) return ST_EINVAL;
    if (d->op == ST_CONVDIFF && !(d->eps > 0)) return ST_EINVAL;
    if (d->kappa < 0) return ST_EINVAL;
    if (d->precision != ST_FP64 && d->precision != ST_MIXED) return ST_EINVAL;
    keep_pool_memory();
    st_problem* p = new st_problem();
    p->d = *d;
    p->d.row_ptr = nullptr;
    p->d.col_idx = nullptr;
    p->d.m_vals = nullptr;
    p->d.a_vals = nullptr;
    if (p->d.tol <= 0) p->d.tol = 1e-8;
    if (p->d.maxit <= 0) p->d.maxit = 400;
    if (p->d.max_basis <= 0) p->d.max_basis = 2048;
    p->stream = (cudaStream_t)d->stream;
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        cudaGetLastError();
        p->device = 0;
    }
    p->n_t = d->n_t;
    p->dt = d->T / d->n_t;
    p->kappa = d->kappa > 0 ? d->kappa : 1.0;
    int st = d->dim == 0 ? setup_user_csr(p, *d) : setup_tensor(p);
    if (st == ST_OK) {
        cudaError_t e = cudaStreamSynchronize(p->stream);
        if (e != cudaSuccess) {
            st_note_cuda(e, "setup sync", __FILE__, __LINE__);
            st = ST_ECUDA;
        }
    }
    if (st != ST_OK) {
        st_destroy(p);
        return st;
    }
    *out = p;
    return ST_OK;
}

extern "C" int st_problem_info(const st_problem* p, int* n_h, int* n_t, int* nnz, double* dt) {
    if (!p) return ST_EINVAL;
    if (n_h) *n_h = p->n_h;
    if (n_t) *n_t = p->n_t;
    if (nnz) *nnz = p->nnz;
    if (dt) *dt = p->dt;
    return ST_OK;
}

extern "C" int st_get_csr(st_problem* p, int* row_ptr, int* col_idx, double* m_vals, double* a_vals) {
    if (!p) return ST_EINVAL;
    if (row_ptr) ST_CUDA_TRY(cudaMemcpyAsync(row_ptr, p->row_ptr, sizeof(int) * (p->n_h + 1), cudaMemcpyDeviceToHost, p->stream));
    if (col_idx) ST_CUDA_TRY(cudaMemcpyAsync(col_idx, p->col, sizeof(int) * p->nnz, cudaMemcpyDeviceToHost, p->stream));
    if (m_vals) ST_CUDA_TRY(cudaMemcpyAsync(m_vals, p->m64, sizeof(double) * p->nnz, cudaMemcpyDeviceToHost, p->stream));
    if (a_vals) ST_CUDA_TRY(cudaMemcpyAsync(a_vals, p->a64, sizeof(double) * p->nnz, cudaMemcpyDeviceToHost, p->stream));
    ST_CUDA_TRY(cudaStreamSynchronize(p->stream));
    return ST_OK;
}

// ---------------------------------------------------------------------------
// Manufactured loads (Section 3, eq. par2) with exact integrals:
// (sin(w x), phi_i) = sin(w x_i) * 2 (1 - cos(w h)) / (h w^2), w = pi/L,
// (pi cos(pi t), tau^l) = sin(pi t^l) - sin(pi t^{l-1}),
// (c sin(pi t), tau^l) = c (cos(pi t^{l-1}) - cos(pi t^l)) / pi.
// Differences of sines and cosines are written as products to avoid
// cancellation for small dt.
// ---------------------------------------------------------------------------
__global__ void k_manufactured_space(int dim, int nx, int ny, int nz, double Lx, double Ly, double Lz,
                                     double* __restrict__ F1, int ldf1, int n_h) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_h) return;
    int idx[3] = {r % nx, (r / nx) % ny, r / (nx * ny)};
    int nn[3] = {nx, ny, nz};
    double L[3] = {Lx, Ly, Lz};
    double g = 1.0;
    for (int d = 0; d < dim; ++d) {
        double h = L[d] / (nn[d] + 1);
        double w = M_PI / L[d];
        double s = sinpi((double)(idx[d] + 1) / (double)(nn[d] + 1));
        double half = sinpi(0.5 * h / L[d]);
        g *= s * (4.0 * half * half) / (h * w * w);
    }
    F1[r] = g;
    F1[r + (size_t)ldf1] = g;
}

__global__ void k_manufactured_time(int n_t, double dt, double c_b, double* __restrict__ F2, int ldf2) {
    int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n_t) return;
    double a = (l + 1) * dt, b = l * dt;
    double mid = 0.5 * (a + b), hw = 0.5 * (a - b);
    double sh = sinpi(hw);
    F2[l] = 2.0 * cospi(mid) * sh;                     // sin(pi a) - sin(pi b)
    F2[l + (size_t)ldf2] = c_b * 2.0 * sinpi(mid) * sh / M_PI;  // c_b (cos(pi b) - cos(pi a)) / pi
}

extern "C" int st_rhs_manufactured(st_problem* p, double* F1, int ldf1, double* F2, int ldf2) {
    if (!p || !F1 || !F2) return ST_EINVAL;
    if (p->dim == 0 || p->d.op != ST_HEAT) return ST_ENOTSUP;
    if (ldf1 < p->n_h || ldf2 < p->n_t) return ST_EINVAL;
    double cb = 0.0;
    for (int d = 0; d < p->dim; ++d) cb += (M_PI / p->len[d]) * (M_PI / p->len[d]);
    cb *= p->kappa;
    k_manufactured_space<<<(p->n_h + 255) / 256, 256, 0, p->stream>>>(p->dim, p->n[0], p->n[1], p->n[2], p->len[0],
                                                                       p->len[1], p->len[2], F1, ldf1, p->n_h);
    ST_LAUNCH_CHECK();
    k_manufactured_time<<<(p->n_t + 255) / 256, 256, 0, p->stream>>>(p->n_t, p->dt, cb, F2, ldf2);
    ST_LAUNCH_CHECK();
    return ST_OK;
}
