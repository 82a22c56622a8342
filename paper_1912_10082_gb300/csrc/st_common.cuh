// Internal declarations shared by the library's translation units.
#pragma once

#include <atomic>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <thread>
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <vector>

#include "st.h"

#define ST_CUDA_TRY(expr)                                   \
    do {                                                    \
        cudaError_t e__ = (expr);                           \
        if (e__ != cudaSuccess) { st_note_cuda(e__, #expr, __FILE__, __LINE__); return ST_ECUDA; } \
    } while (0)

#define ST_LAUNCH_CHECK()                                   \
    do {                                                    \
        st_count_launch();                                  \
        cudaError_t e__ = cudaGetLastError();               \
        if (e__ != cudaSuccess) { st_note_cuda(e__, "launch", __FILE__, __LINE__); return ST_ECUDA; } \
    } while (0)

#define ST_TRY(expr)                                        \
    do { int s__ = (expr); if (s__ != ST_OK) return s__; } while (0)

void st_note_cuda(cudaError_t e, const char* what, const char* file, int line);
void st_note_msg(const char* msg);   // sets the text returned by st_last_error

// Pinned host buffers taken from and returned to a process-wide pool (st_setup.cu).  Allocating or freeing
// pinned memory, like a synchronous device allocation or free, waits for the whole device, so a solve that
// grew or released its staging this way would stall every other solve running on the GPU.  st_pinned_get
// returns at least `bytes` (the size in *got) or nullptr; st_pinned_put takes a buffer back once no copy
// in flight uses it.  Pooled buffers stay allocated for the life of the process.
void* st_pinned_get(size_t bytes, size_t* got);
void st_pinned_put(void* ptr, size_t bytes);

// launch accounting and optional event timing (st_profile.cu)
void st_count_launch();
void st_count_launches(unsigned long long n);
void st_capture_enter();
void st_capture_leave();
void st_prof_begin(cudaStream_t s, const char* tag, double bytes, double flops);
void st_prof_end(cudaStream_t s);

// Launch-variant tuning (st_tune.h).  While a session is set on the calling
// thread, a launcher whose shape is missing from the table times each valid
// variant on the launch's own operands, records the pick and then launches it.
struct StTuneSession {
    void* scratch = nullptr;   // device bytes for saving the input of an in-place launch
    size_t scratch_bytes = 0;
    int tuned = 0;             // shapes this session added to the table
};
// Sets the calling thread's session and returns the one it replaces.
StTuneSession* st_tune_set_session(StTuneSession* sess);
// The calling thread's session, or nullptr when none is set or s is being captured.
StTuneSession* st_tune_session(cudaStream_t s);
// Times n launch variants on stream s: run(c) launches variant c (valid[c]
// only); prep, if given, runs before every launch outside the timed span (it
// restores the input of an in-place launch).  Four rounds (the first a
// warm-up) of three launches a variant, interleaved; ms[c] = the best round's
// time, or -1 for an invalid variant.  Synchronises s.
int st_tune_measure(cudaStream_t s, int n, const bool* valid, const std::function<void(int)>& run,
                    const std::function<int()>& prep, double* ms);

// One device allocation owned by a handle.
struct DevArray {
    void* ptr = nullptr;
    size_t bytes = 0;
};

// 1D factors of one box direction for the fast-diagonalisation solve.
struct FdAxis {
    int n = 0;
    double h = 0.0;         // mesh width L/(n+1)
    double* Q64 = nullptr;  // n x n, Q[j][i] = sin((j+1)(i+1) pi/(n+1)), symmetric
    float* Q32 = nullptr;
    double* lam = nullptr;  // eigenvalues of K phi = lam M phi, j = 1..n
    double* c2 = nullptr;   // 2 / ((n+1) mu_j), mu_j the M eigenvalue of sine mode j
    float* lam32 = nullptr; // the same in FP32 (FP32 epilogues stay off the FP64 pipe)
    float* c232 = nullptr;
    // folded half tables {H0, H1, G0, G1}: H_p[k][i'] = Q[k][2i'+p] (k, i' < K_p, K_0 = ceil(n/2),
    // K_1 = floor(n/2)), G_p = H_p^T
    double* fold64[4] = {};
    float* fold32[4] = {};
};

struct st_problem {
    st_desc d{};
    cudaStream_t stream = nullptr;
    int device = 0;         // CUDA device current at st_setup (owner of every buffer)
    int dim = 0;            // 0 for user CSR
    int n[3] = {1, 1, 1};
    double len[3] = {1, 1, 1};
    int n_h = 0, n_t = 0, nnz = 0, max_row_nnz = 0;
    double dt = 0.0, kappa = 1.0;
    bool tensor_heat = false;   // fast-diagonalisation solver applies
    // CSR, shared pattern (device)
    int* row_ptr = nullptr;
    int* col = nullptr;
    double *m64 = nullptr, *a64 = nullptr, *p64 = nullptr, *q64 = nullptr;   // M, A, P=M+dt/2A, N=M-dt/2A
    double* at64 = nullptr;     // A^T on the same (symmetric) pattern; box problems only
    float *m32 = nullptr, *a32 = nullptr, *p32 = nullptr, *q32 = nullptr;
    FdAxis ax[3];
    // stencil of P and N on a box grid (every n_d >= 3): the 27 values of an interior
    // row in (dz, dy, dx) order, copied from the assembled CSR (zeros beyond dim)
    bool box_ok = false;
    double box_p64[27] = {}, box_q64[27] = {};
    float box_p32[27] = {}, box_q32[27] = {};
    double box_m64[27] = {}, box_a64[27] = {};   // M and A (Aᵀ = A reversed) for the spatial products
    float box_m32[27] = {}, box_a32[27] = {};
    // x-line preconditioner of convection-diffusion: Thomas factors of
    // eps Kx + beta_x Gx + mu Mx for every mode of the transformed directions,
    // for the shift line_shift (n_h entries each)
    double *line_cp64 = nullptr, *line_ip64 = nullptr;
    float *line_cp32 = nullptr, *line_ip32 = nullptr;
    double line_shift = -1.0;
    bool line_valid = false;
    double lam_min = 0.0, lam_max = 0.0;   // spectrum of the pencil (A, M), or of its diffusion part
    double fd_lam_min = 0.0, fd_lam_max = 0.0;   // the same for unit diffusion (sums of 1D sine-mode eigenvalues)
    double fd_kappa = 1.0;                 // diffusion the fast-diagonalisation transforms use
    std::vector<void*> owned;              // every device allocation of the handle
    // solution of the last st_solve (device, owned)
    double* V = nullptr;
    float2* Vdf = nullptr;      // double-float copy of V (mixed precision), same capacity
    double* Y = nullptr;
    int k = 0;
    size_t V_cap_cols = 0, Y_cap = 0;
    // persistent solver workspace (device, owned), grown on demand
    double* work = nullptr;
    size_t work_bytes = 0;
    // CN graph cache
    void* cn_graph = nullptr;   // cudaGraphExec_t
    bool cn_stale = false;      // coefficients changed since the capture: recapture and update
    size_t cn_nodes = 0;        // kernel nodes in the CN graph
    double* cn_buf = nullptr;
    const void* cn_key[4] = {nullptr, nullptr, nullptr, nullptr};
    // grow-only device workspace slots
    void* slot_ptr[32] = {};
    size_t slot_bytes[32] = {};
    // staging area of the solver's synchronisation points: sm_dev holds
    // [download region | upload region] of sm_cap doubles each on the device,
    // sm_host the pinned host mirror of both
    double* sm_dev = nullptr;
    double* sm_host = nullptr;
    size_t sm_cap = 0;
    size_t sm_host_bytes = 0;   // size of the pooled pinned buffer behind sm_host
};

// Returns a device buffer of at least `bytes` for slot `id` (contents not kept on growth).
int st_slot(st_problem* p, int id, size_t bytes, void** out);

// ---- allocation helpers (st_setup.cu) ----
int st_alloc(st_problem* p, void** ptr, size_t bytes);
int st_free_one(st_problem* p, void* ptr);
bool st_is_device_ptr(const void* ptr);
// Copies a possibly-host column-major matrix into a device buffer with ld = rows.
int st_stage_matrix(st_problem* p, const double* src, int ld, int rows, int cols, double* dst);

// ---- kernels launched from several files (st_kernels.cu) ----
// Out1 = M X, Out2 = A X for ncols columns (either output may be NULL).
template <typename T>
int st_spmm_ma(st_problem* p, const T* X, int ldx, int ncols, T* OutM, int ldm, T* OutA, int lda, cudaStream_t s);
// Out = A^T X (box problems: A^T is stored on the shared pattern)
int st_spmm_at64(st_problem* p, const double* X, int ldx, int ncols, double* Out, int ldo, cudaStream_t s);
// Out = alpha * (Mv * M + Av * A) X + beta * Out
int st_spmm_comb64(st_problem* p, double cm, double ca, const double* X, int ldx, int ncols,
                   double beta, double* Out, int ldo, cudaStream_t s);
// Space-time apply Y[:,l] = P u_l - N u_{l-1}.
template <typename T>
int st_apply_kernel(st_problem* p, const T* U, int ldu, T* Y, int ldy, int n_t, cudaStream_t s);
// Right-hand side of CN step l: out = N u + F1 F2[l, :]^T; u may be NULL (u_0 = 0).
int st_cn_rhs_step(st_problem* p, const double* u, const double* F1, int ldf1, const double* F2, int ldf2, int l,
                   int ncols, double* out, cudaStream_t s);

// Fast-diagonalisation transform: W = coef * Q (x) diag(omega) Q (x) X with
// omega(j) = weight(j) / (kappa * sum lam + shift), weight = prod c2 (kind 1) or 1 (kind 0).
enum FdKind { FD_MASS_RESOLVENT = 0, FD_RESOLVENT = 1, FD_MASS_INVERSE = 2 };
int st_fd_apply64(st_problem* p, FdKind kind, double shift, double coef, const double* X, int ldx,
                  int ncols, double* W, int ldw, double* tmp, cudaStream_t s);
// Constant box stencils of two spatial operators (27 values each, (dz, dy, dx)
// order, zeros beyond the grid's dimension), passed to the box-stencil kernels.
template <typename T>
struct BoxPair {
    T s[2][27];
};

// 1D factors of a box problem's M and A (the sum-factorised apply): per
// direction d the mass stencil (m1, m0, m1) and the operator stencil
// (am, a0, ap) on the offsets (-1, 0, +1); hdt = dt / 2.
struct SfStencil {
    float m0[3], m1[3];
    float am[3], a0[3], ap[3];
    float hdt;
};

// Epilogue of a fast-diagonalisation mode product: a constant factor and,
// for the middle product, the spectral weight of the output entry.
struct FdEpi {
    int scale;          // 0: C = coef * acc; 1: C = coef * omega(e) * acc
    int left;           // 1: linear index e = m * J + j (batch = one vector column); 0: e = m
    long long J;
    int dim, nx, ny, nz;
    const double *l0, *l1, *l2;   // eigenvalues per direction
    const double *c0, *c1, *c2;   // c2 factors per direction (resolvent of a general right-hand side)
    const float *f0, *f1, *f2;    // FP32 copies of l0..l2 and of c0..c2, for FP32 products
    const float *g0, *g1, *g2;
    int kind;           // FdKind
    double kappa, shift, coef;
};

// Batch index z = blockIdx.z splits into (z2, z1) = (z / nb1, z % nb1); the
// operand offsets are z1 * s*1 + z2 * s*2.
struct Batch2 {
    int nb1;
    long long sA1, sA2, sB1, sB2, sC1, sC2;
};

// x-line preconditioner (convection-diffusion with |beta_x| the largest
// component): W = coef (eps K + beta_x Gx (x) M_rest + s M)^{-1} X, exact in
// 1D; y (and z) by sine transforms, x by Thomas sweeps with the factors of
// st_line_factor (call it for the shift first).
bool st_line_usable(const st_problem* p);
int st_line_factor(st_problem* p, double shift, cudaStream_t s);
int st_line_apply64(st_problem* p, double coef, const double* X, int ldx, int ncols, double* W, int ldw, double* tmp,
                    cudaStream_t s);
int st_line_apply32(st_problem* p, double coef, const float* X, int ldx, int ncols, float* W, int ldw, float* tmp,
                    cudaStream_t s);
int st_fd_apply32(st_problem* p, FdKind kind, double shift, double coef, const float* X, int ldx,
                  int ncols, float* W, int ldw, float* tmp, cudaStream_t s);

// Tall-skinny products.  H (k x m, ld ldh, device) = V^T W for V n x k, W n x m.
// partial must hold tsgemm_partial_elems(n, k, m) doubles.
size_t st_tsgemm_partial_elems(int n, int k, int m);
// batched flexible GMRES (m independent Arnoldi processes, vectors interleaved)
size_t st_gm_partial_elems(int n, int kk, int m);
template <typename T>
int st_gm_dots(int n, int kk, int m, const T* Z, double* part, double* H, int ldh, cudaStream_t s);
template <typename T>
int st_gm_update(int n, int nb, int m, T* Z, const double* H, int ldh, const double* H1, int ldh1, double* Hd,
                 long long ldhd, int jcol, int J, cudaStream_t s);
template <typename T>
int st_gm_update_dot(int n, int nb, int m, T* Z, const double* H1, int ldh1, double* part, double* H2, int ldh2,
                     cudaStream_t s);
int st_scale_cols_to32(int n, int m, const double* X, int ldx, const double* f, float* Y, int ldy, cudaStream_t s);
struct GmSteps {   // Arnoldi steps that enter each column's solution (at most 16 columns)
    int v[16];
};
int st_gm_accumulate32(int n, int m, const float* T, const double* y, int ldy, const GmSteps& ju, double* W, int ldw,
                       cudaStream_t s);
int st_spmm_comb32(st_problem* p, double cm, double ca, const float* X, int ldx, int ncols, float* Out, int ldo,
                   cudaStream_t s);
int st_scale_cols_dev(int n, int m, double* X, int ldx, const double* f, cudaStream_t s);
int st_tsgemm_tn(int n, int k, int m, const double* V, int ldv, const double* W, int ldw,
                 double* H, int ldh, double* partial, cudaStream_t s);
// W = beta * W + alpha * V H   (V n x k, H k x m device, W n x m)
int st_tsgemm_nn(int n, int k, int m, double alpha, const double* V, int ldv, const double* H, int ldh,
                 double beta, double* W, int ldw, cudaStream_t s);
// Double-float variants for a basis V stored as (hi, lo) float pairs: FP64-accurate
// to about 48 bits, computed on the FP32 pipes.
int st_to_df(int n, int m, const double* X, int ldx, float2* Y, int ldy, cudaStream_t s);
// hi_only: the FP32 product of the leading parts (first pass of the block Gram-Schmidt).
int st_tsgemm_tn_df(int n, int k, int m, const float2* V, int ldv, const float2* W, int ldw,
                    double* H, int ldh, double* partial, cudaStream_t s, bool hi_only = false);
int st_tsgemm_nn_df(int n, int k, int m, double alpha, const float2* V, int ldv, const double* H, int ldh,
                    double beta, double* W, int ldw, cudaStream_t s);
// W = W * R^{-1} for upper triangular R (m x m, device), in place
int st_trsm_right_upper(int n, int m, const double* R, int ldr, double* W, int ldw, cudaStream_t s);
// R (upper, m x m, ld ldr, device) with R^T R = G (m x m, ld ldg, device), m <= 16, by one warp.
// On a non-positive pivot *flag (device) is set to 1 and R to the identity; else *flag = 0.
int st_chol_small(int m, const double* G, int ldg, double* R, int ldr, double* flag, cudaStream_t s);

// small vector helpers
int st_copy_cols64(int n, int m, const double* X, int ldx, double* Y, int ldy, cudaStream_t s);
int st_convert_64_32(int n, int m, const double* X, int ldx, float* Y, int ldy, cudaStream_t s);
int st_convert_32_64_add(int n, int m, const float* X, int ldx, double* Y, int ldy, double beta, cudaStream_t s);
int st_axpby64(int n, int m, double a, const double* X, int ldx, double b, double* Y, int ldy, cudaStream_t s);
// C = X Y, all column-major (r x c = r x s times s x c), FP64.
int st_gemm_cm(int r, int c, int s, const double* X, int ldx, const double* Y, int ldy, double* C, int ldc,
               cudaStream_t st);
int st_lowrank_dense(int n, int k, int n_t, const double* V, int ldv, const double* Y, int ldy,
                     double* U, int ldu, cudaStream_t s);

// ---- host dense algebra (st_dense.cpp), column-major, FP64 ----
// Host threads for the projected problems (st_dense.cpp).  Parallel loops
// give each output element to one thread and keep its serial summation order,
// so results do not depend on the thread count.
namespace hostpar {
struct ActiveSolve {   // counts solves in flight; they share the host cores
    ActiveSolve();
    ~ActiveSolve();
};
int threads_for(double flops);   // 1 .. 8 threads for a job of this size
class Barrier {
   public:
    explicit Barrier(int count) : n(count) {}
    void wait();

   private:
    std::atomic<int> arrived{0};
    std::atomic<unsigned> gen{0};
    int n;
};
void run(int T, const std::function<void(int, Barrier&)>& body);   // body(t, barrier), t = 0 on the caller
// While a ThreadBudget lives on a thread, threads_for() returns at most n
// there: work already spread over a Pool's threads starts thread teams of at
// most its share of the cores (n = 1: none).
struct ThreadBudget {
    explicit ThreadBudget(int n);
    ~ThreadBudget();
    int prev;
};
// Persistent worker threads for loops over independent items (the instances
// of a batched solve).  run(n, f) calls f(i) for every i in [0, n) on the
// workers and the caller, each item on one thread, and returns when all are
// done.  Each item runs under a ThreadBudget of max(1, threads / n), so a few
// large items still use the cores.  Not reentrant.
class Pool {
   public:
    explicit Pool(int threads);   // total threads including the caller, >= 1
    ~Pool();
    void run(int n, const std::function<void(int)>& f);
    int threads() const { return (int)workers_.size() + 1; }

   private:
    void work();
    std::vector<std::thread> workers_;
    std::mutex mu_;
    std::condition_variable cv_, done_cv_;
    const std::function<void(int)>* job_ = nullptr;
    std::atomic<int> next_{0};
    int n_ = 0, busy_ = 0;
    unsigned gen_ = 0;
    bool stop_ = false;
};
}  // namespace hostpar

namespace dense {
bool cholesky(int n, double* A, int lda);                 // lower, in place
void chol_solve(int n, const double* L, int ldl, double* B, int ldb, int nrhs);
void lower_solve(int n, const double* L, int ldl, double* B, int ldb, int nrhs);   // L X = B
bool lu(int n, double* A, int lda, int* piv);
void lu_solve(int n, const double* LU, int lda, const int* piv, double* B, int ldb, int nrhs);
bool lu_solve_transpose(int n, const double* LU, int lda, const int* piv, double* B, int ldb, int nrhs);
void sym_eigvals(int n, double* A, int lda, double* w);   // destroys A, ascending w
void sym_eig(int n, double* A, int lda, double* w);       // A <- eigenvectors (columns), ascending w
int  thin_qr(int m, int n, double* A, int lda, double* R, int ldr); // Householder, A <- Q
void svd_small(int m, int n, const double* A, int lda, double* U, double* s, double* Vt); // m, n small
}  // namespace dense
