// Grouped launches for the batched solve (st_solve_batch): one launch of a
// kernel serves the same step of every instance of a batch.  Each instance
// contributes one or more tasks; a task is split into tiles (the CTAs the
// single-problem kernel would launch for it), and a persistent grid walks the
// concatenated tile list, finding each tile's task by binary search in a
// prefix array.  The tile bodies are those of the single-problem kernels
// (st_dev.cuh), so a grouped step computes exactly what the single-problem
// launches compute, instance by instance.
//
// Host side: a GroupPhase collects the tasks of consecutive grouped launches
// into one pinned staging buffer, copies it to the device in one transfer and
// then issues the launches in order on one stream.
#pragma once

#include <functional>
#include <vector>

#include "st_common.cuh"

namespace stg {

// Mode product of the fast-diagonalisation transform (k_gemm_fold's tile body).
struct FoldTask {
    int n, other;
    const void* X;
    long long ldx;
    const void* HG[4];
    void* C;
    long long ldc;
    Batch2 bt;
    FdEpi ep;
    int gx, gy, gz;   // tiles: gx * gy * gz (gz = 2 * batch: both parities)
    int tc;           // FP32 only: 1 = tensor-core tiles (128 x 128), 0 = SIMT tiles
    int tm;           // SIMT tiles: 16 tm x 16 tm outputs (tm 2, or 4 for the FP32 vector-read tile)
};

// Box-stencil product O1 = S1 X (+ beta O1), O2 = S2 X (k_stencil_box's tile body, FP64).
struct StencilTask {
    int nx, ny, nz;
    BoxPair<double> S;
    const double* X;
    long long ldx;
    double beta;
    double* O1;
    long long ld1;
    double* O2;
    long long ld2;
    int blocks, ncols;   // tiles: blocks * ncols
};

// H = V^T W over n rows: chunk partials then their fixed-order sum (FP64, or
// double-float V, W with float2 partials).  At most 16 columns of W a task.
struct TnTask {
    int n, k, m, rows, nch;   // rows per chunk (ts_rows), chunks
    const void* V;
    long long ldv;
    const void* W;
    long long ldw;
    void* part;               // nch * k * m partials (doubles, or float2 pairs in the same room)
    double* H;
    long long ldh;
};

// W = beta W + alpha V H (FP64 V, or double-float V), at most 16 columns a task.
struct NnTask {
    int n, k, m;
    double alpha;
    const void* V;
    long long ldv;
    const double* H;
    long long ldh;
    double beta;
    double* W;
    long long ldw;
};

// W <- W R^{-1} (R upper, m x m <= 16 x 16).
struct TrsmTask {
    int n, m;
    const double* R;
    long long ldr;
    double* W;
    long long ldw;
};

// R^T R = G by one warp (m <= 16); *flag = 1 on a non-positive pivot.
struct CholTask {
    int m;
    const double* G;
    long long ldg;
    double* R;
    long long ldr;
    double* flag;
};

// Column-wise elementwise operations on n x m blocks.
enum ElemOp {
    E_COPY64 = 0,   // Y = X (double)
    E_TO32 = 1,     // Y = (float) X
    E_ADD32 = 2,    // Y = (double) X + b Y  (X float; the term b Y only when b != 0)
    E_AXPBY = 3,    // Y = a X + b Y (double; b Y only when b != 0)
    E_TO_DF = 4     // Y = (hi, lo) split of X (float2)
};
struct ElemTask {
    int op, n, m;
    const void* X;
    long long ldx;
    void* Y;
    long long ldy;
    double a, b;
};

// Pinned staging buffer and its device copy for the task tables of one
// stream's grouped launches (owned by the caller).  Runs append to it; the
// caller calls reset() only when the stream has passed every earlier run
// (right after a synchronisation), so a table is never overwritten while a
// copy or a launch may still read it.
struct GroupArena {
    char* h = nullptr;   // pinned, from the library's pool
    char* d = nullptr;   // stream-ordered
    size_t cap = 0, used = 0, hbytes = 0;
    cudaStream_t s_ = nullptr;
    ~GroupArena();
    // Room for `bytes` more; when the buffers must grow, synchronises s first
    // (everything earlier has then run, so the new buffers start empty).
    int reserve(size_t bytes, cudaStream_t s);
    void reset() { used = 0; }
};

class GroupPhase {
   public:
    GroupPhase(cudaStream_t s, GroupArena* arena) : s_(s), arena_(arena) {}
    // Each add_* queues one grouped launch (skipped when it has no task).
    void fold(int tsize, int side, const std::vector<FoldTask>& t);   // tsize 4 (float) or 8 (double)
    void fold_tc(int side, const std::vector<FoldTask>& t);           // FP32 tasks on the tensor cores
    void fold_simt(int tsize, int side, int tm, const std::vector<FoldTask>& t);
    void stencil(int dim, const std::vector<StencilTask>& t);
    // partials and their sums: two launches; hi: the FP32 product of the double-float leading parts
    void tn(bool df, const std::vector<TnTask>& t, bool hi = false);
    void nn(bool df, const std::vector<NnTask>& t);
    void trsm(const std::vector<TrsmTask>& t);
    void chol(const std::vector<CholTask>& t);
    void elem(const std::vector<ElemTask>& t);
    // Copies every queued task table to the device (one transfer into the
    // arena) and issues the launches in queue order on the stream.  The phase
    // is empty afterwards and can queue the next launches.
    int run();
    int launches() const { return launches_; }

   private:
    struct Pending {
        std::function<void(const char* dev_base)> go;
        const char* tag = nullptr;   // profiling record (st_profile_*) opened before this launch, or none
        double bytes = 0.0, flops = 0.0;
        bool close = true;           // the record ends after this launch
    };
    size_t put(const void* p, size_t bytes);
    template <class Task>
    size_t put_tasks(const std::vector<Task>& t, const std::vector<int>& tiles, int* total);
    cudaStream_t s_;
    GroupArena* arena_;
    std::vector<char> host_;
    std::vector<Pending> pend_;
    int launches_ = 0;
};

}  // namespace stg
