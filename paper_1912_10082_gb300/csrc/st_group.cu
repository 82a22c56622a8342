// Grouped kernels of the batched solve: one launch serves one step of every
// instance of a batch (see st_group.h).  Each kernel is a persistent loop over
// the tiles of all its tasks; a tile runs the tile body of the single-problem
// kernel (st_dev.cuh) with the task's operands.
#include <algorithm>
#include <cstring>

#include "st_common.cuh"
#include "st_dev.cuh"
#include "st_group.h"

namespace {

constexpr int kMaxGrid = 152 * 24;   // persistent grid: at most 24 CTAs per SM in flight or queued
constexpr int kSub = 8;              // row blocks of 256 per tile of the elementwise and triangular kernels

// Task index of tile t: the largest i with prefix[i] <= t.
__device__ __forceinline__ int g_task(const int* __restrict__ prefix, int ntasks, int t) {
    int lo = 0, hi = ntasks - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(prefix + mid) <= t)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Cooperative copy of a task record into shared memory (every field is 4 or 8 bytes).
template <class Task>
__device__ __forceinline__ void g_load(Task& dst, const Task* src, int tid, int nthr) {
    static_assert(sizeof(Task) % 4 == 0, "task records are made of 4- and 8-byte fields");
    const int* s = reinterpret_cast<const int*>(src);
    int* d = reinterpret_cast<int*>(&dst);
    for (int w = tid; w < (int)(sizeof(Task) / 4); w += nthr) d[w] = __ldg(s + w);
}

// FP32 64 x 64 tiles: four CTAs an SM (64 registers; the x-direction tile spills a few words, still faster
// than three CTAs without spills)
template <typename T, int TM, int SIDE>
__global__ void __launch_bounds__(256, TM == 4 && sizeof(T) == 4 ? 4 : 3) kg_fold(const stg::FoldTask* tasks, const int* prefix,
                                                               int ntasks) {
    __shared__ stg::FoldTask tk;
    const int total = prefix[ntasks];
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int i = g_task(prefix, ntasks, t);
        __syncthreads();   // the previous tile is done with tk and with the body's shared tiles
        g_load(tk, tasks + i, threadIdx.x, 256);
        __syncthreads();
        int local = t - prefix[i];
        const int bx = local % tk.gx;
        local /= tk.gx;
        const int by = local % tk.gy, bz = local / tk.gy;
        fold_tile<T, TM, SIDE>(tk.n, tk.other, (const T*)tk.X, tk.ldx, (const T*)tk.HG[0], (const T*)tk.HG[1],
                                    (const T*)tk.HG[2], (const T*)tk.HG[3], (T*)tk.C, tk.ldc, tk.bt, tk.ep, bx, by,
                                    bz);
    }
}

// Tensor-core mode products (FP32): TMEM allocated once per CTA, one mbarrier whose phase runs across
// the tiles; a tile whose MMA wait gave up stops the CTA (its outputs are NaN, see fold_tc_body).
template <int SIDE>
__global__ void __launch_bounds__(FTC_THREADS, 1) kg_fold_tc(const stg::FoldTask* tasks, const int* prefix,
                                                            int ntasks) {
    extern __shared__ __align__(1024) unsigned char ftc_sm[];
    __shared__ stg::FoldTask tk;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tslot;
    ftc_alloc(&tslot);
    ftc_mbar_init(&mbar);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    uint32_t ph = 0;
    const int total = prefix[ntasks];
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int i = g_task(prefix, ntasks, t);
        __syncthreads();
        g_load(tk, tasks + i, threadIdx.x, FTC_THREADS);
        __syncthreads();
        int local = t - prefix[i];
        const int bx = local % tk.gx;
        local /= tk.gx;
        const int by = local % tk.gy, bz = local / tk.gy;
        if (!fold_tc_body<SIDE>(tk.n, tk.other, (const float*)tk.X, tk.ldx, (const float*)tk.HG[2],
                                (const float*)tk.HG[3], (float*)tk.C, tk.ldc, tk.bt, tk.ep, bx, by, bz, ftc_sm, tslot,
                                &mbar, &ph))
            break;   // uniform: every thread of the CTA saw the same waits
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    ftc_dealloc(tslot);
}

// 2D: three CTAs an SM (80 registers instead of 86 and two CTAs; 54 -> 47 ms in the 256-problem batch)
template <int DIM>
__global__ void __launch_bounds__(256, DIM == 2 ? 3 : 1) kg_stencil(const stg::StencilTask* tasks, const int* prefix, int ntasks) {
    __shared__ stg::StencilTask tk;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int total = prefix[ntasks];
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int i = g_task(prefix, ntasks, t);
        __syncthreads();
        g_load(tk, tasks + i, tid, 256);
        __syncthreads();
        const int local = t - prefix[i];
        stencil_box_body<double, DIM, 2, DIM == 2 ? 1 : 2>(tk.nx, tk.ny, tk.nz, tk.S, tk.X, tk.ldx, tk.beta, tk.O1,
                                                           tk.ld1, tk.O2, tk.ld2, local % tk.blocks,
                                                           local / tk.blocks);
    }
}

template <int MAXM, bool DF, bool HI = false>
__global__ void __launch_bounds__(TS_THREADS, 4) kg_tn_partial(const stg::TnTask* tasks, const int* prefix, int ntasks) {
    extern __shared__ double smem[];
    __shared__ stg::TnTask tk;
    const int total = prefix[ntasks];
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int i = g_task(prefix, ntasks, t);
        __syncthreads();
        g_load(tk, tasks + i, threadIdx.x, TS_THREADS);
        __syncthreads();
        const int local = t - prefix[i];
        const int bx = local % tk.nch, by = local / tk.nch;
        if constexpr (DF)
            ts_tn_df_partial_body<MAXM, HI>(tk.n, tk.k, tk.m, tk.rows, (const float2*)tk.V, tk.ldv, (const float2*)tk.W,
                                        tk.ldw, (float2*)tk.part, smem, bx, by);
        else
            ts_tn_partial_body<MAXM>(tk.n, tk.k, tk.m, tk.rows, (const double*)tk.V, tk.ldv, (const double*)tk.W,
                                     tk.ldw, (double*)tk.part, smem, bx, by);
    }
}

template <bool DF>
__global__ void __launch_bounds__(256) kg_tn_reduce(const stg::TnTask* tasks, const int* prefix, int ntasks) {
    __shared__ stg::TnTask tk;
    const int total = prefix[ntasks];
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int i = g_task(prefix, ntasks, t);
        __syncthreads();
        g_load(tk, tasks + i, threadIdx.x, 256);
        __syncthreads();
        const int local = t - prefix[i];
        if constexpr (DF)
            ts_reduce_df_body(tk.nch, tk.k, tk.m, (const float2*)tk.part, tk.H, tk.ldh, local);
        else
            ts_reduce_body(tk.nch, tk.k, tk.m, (const double*)tk.part, tk.H, tk.ldh, local);
    }
}

template <int MAXM, bool DF>
__global__ void __launch_bounds__(256) kg_nn(const stg::NnTask* tasks, const int* prefix, int ntasks) {
    __shared__ stg::NnTask tk;
    const int total = prefix[ntasks];
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int i = g_task(prefix, ntasks, t);
        __syncthreads();
        g_load(tk, tasks + i, threadIdx.x, 256);
        __syncthreads();
        const int local = t - prefix[i];
        if constexpr (DF)
            ts_nn_df_body<MAXM>(tk.n, tk.k, tk.m, tk.alpha, (const float2*)tk.V, tk.ldv, tk.H, tk.ldh, tk.beta, tk.W,
                                tk.ldw, local);
        else
            ts_nn_body<MAXM>(tk.n, tk.k, tk.m, tk.alpha, (const double*)tk.V, tk.ldv, tk.H, tk.ldh, tk.beta, tk.W,
                             tk.ldw, local);
    }
}

// three CTAs an SM (80 registers instead of 95, a few spilled words; 36 -> 32 ms in the 256-problem batch)
__global__ void __launch_bounds__(256, 3) kg_trsm(const stg::TrsmTask* tasks, const int* prefix, int ntasks) {
    __shared__ stg::TrsmTask tk;
    const int total = prefix[ntasks];
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int i = g_task(prefix, ntasks, t);
        __syncthreads();
        g_load(tk, tasks + i, threadIdx.x, 256);
        __syncthreads();
        // kSub row blocks of 256 a tile (fewer task look-ups and barriers per row)
        for (int sb = 0; sb < kSub; ++sb) {
            if (sb) __syncthreads();   // the previous block is done reading R from shared memory
            trsm_right_upper_body(tk.n, tk.m, tk.R, tk.ldr, tk.W, tk.ldw, (t - prefix[i]) * kSub + sb);
        }
    }
}

__global__ void __launch_bounds__(32) kg_chol(const stg::CholTask* tasks, const int* prefix, int ntasks) {
    __shared__ stg::CholTask tk;
    const int total = prefix[ntasks];
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int i = g_task(prefix, ntasks, t);
        __syncwarp();
        g_load(tk, tasks + i, threadIdx.x, 32);
        __syncwarp();
        chol_small_body(tk.m, tk.G, tk.ldg, tk.R, tk.ldr, tk.flag);
    }
}

__global__ void __launch_bounds__(256) kg_elem(const stg::ElemTask* tasks, const int* prefix, int ntasks) {
    __shared__ stg::ElemTask tk;
    const int total = prefix[ntasks];
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int i = g_task(prefix, ntasks, t);
        __syncthreads();
        g_load(tk, tasks + i, threadIdx.x, 256);
        __syncthreads();
        for (int sb = 0; sb < kSub; ++sb) {   // kSub blocks of 256 entries a tile
            const int local = (t - prefix[i]) * kSub + sb;
            switch (tk.op) {
                case stg::E_COPY64:
                    copy_cols_body<double, double>(tk.n, tk.m, (const double*)tk.X, tk.ldx, (double*)tk.Y, tk.ldy, 0.0,
                                                   local);
                    break;
                case stg::E_TO32:
                    copy_cols_body<double, float>(tk.n, tk.m, (const double*)tk.X, tk.ldx, (float*)tk.Y, tk.ldy, 0.0,
                                                  local);
                    break;
                case stg::E_ADD32:
                    copy_cols_body<float, double>(tk.n, tk.m, (const float*)tk.X, tk.ldx, (double*)tk.Y, tk.ldy, tk.b,
                                                  local);
                    break;
                case stg::E_AXPBY:
                    axpby_body(tk.n, tk.m, tk.a, (const double*)tk.X, tk.ldx, tk.b, (double*)tk.Y, tk.ldy, local);
                    break;
                default:
                    to_df_body(tk.n, tk.m, (const double*)tk.X, tk.ldx, (float2*)tk.Y, tk.ldy, local);
                    break;
            }
        }
    }
}

inline int grid_for(int total) { return std::max(1, std::min(total, kMaxGrid)); }

template <class F>
void with_maxm(int m, F&& f) {
    if (m <= 2)
        f(std::integral_constant<int, 2>{});
    else if (m <= 4)
        f(std::integral_constant<int, 4>{});
    else if (m <= 8)
        f(std::integral_constant<int, 8>{});
    else
        f(std::integral_constant<int, 16>{});
}

}  // namespace

namespace stg {

GroupArena::~GroupArena() {
    if (s_) cudaStreamSynchronize(s_);   // the last task-table copies have landed
    if (d) cudaFreeAsync(d, s_);
    st_pinned_put(h, hbytes);
}

// Growth takes a stream-ordered device buffer and a pinned buffer from the library's pool, so it never waits
// for the work of other streams (a synchronous allocation or free would).
int GroupArena::reserve(size_t bytes, cudaStream_t s) {
    if (used + bytes <= cap) return ST_OK;
    ST_CUDA_TRY(cudaStreamSynchronize(s));   // earlier copies and launches may still read h and d
    used = 0;
    if (bytes <= cap) return ST_OK;
    if (d) cudaFreeAsync(d, s);
    st_pinned_put(h, hbytes);
    h = nullptr;
    d = nullptr;
    cap = hbytes = 0;
    s_ = s;
    const size_t want = std::max<size_t>(4 * bytes, 1 << 20);
    h = (char*)st_pinned_get(want, &hbytes);
    cudaError_t e = h ? cudaMallocAsync((void**)&d, want, s) : cudaErrorMemoryAllocation;
    if (e != cudaSuccess) {
        cudaGetLastError();
        st_note_cuda(e, "grouped task tables", __FILE__, __LINE__);
        st_pinned_put(h, hbytes);
        h = nullptr;
        d = nullptr;
        hbytes = 0;
        return ST_ENOMEM;
    }
    cap = want;
    return ST_OK;
}

size_t GroupPhase::put(const void* p, size_t bytes) {
    const size_t off = (host_.size() + 15) & ~size_t(15);
    host_.resize(off + bytes);
    std::memcpy(host_.data() + off, p, bytes);
    return off;
}

// Appends the tasks and their tile prefix (ntasks + 1 ints); returns the
// offset of the tasks, the prefix follows at the returned offset + its size.
template <class Task>
size_t GroupPhase::put_tasks(const std::vector<Task>& t, const std::vector<int>& tiles, int* total) {
    std::vector<int> prefix(t.size() + 1, 0);
    for (size_t i = 0; i < t.size(); ++i) prefix[i + 1] = prefix[i] + tiles[i];
    *total = prefix.back();
    const size_t off = put(t.data(), sizeof(Task) * t.size());
    put(prefix.data(), sizeof(int) * prefix.size());
    return off;
}

#define ST_PREFIX_OF(off, Task, n) ((((off) + sizeof(Task) * (n)) + 15) & ~size_t(15))

void GroupPhase::fold(int tsize, int side, const std::vector<FoldTask>& all) {
    if (all.empty()) return;
    // tensor-core tasks (FP32) in a launch of their own
    std::vector<FoldTask> t2, t4, tct;
    for (const FoldTask& k : all) (tsize == 4 && k.tc ? tct : (tsize == 4 && k.tm == 4 ? t4 : t2)).push_back(k);
    if (!tct.empty()) fold_tc(side, tct);
    if (!t4.empty()) fold_simt(tsize, side, 4, t4);
    if (!t2.empty()) fold_simt(tsize, side, 2, t2);
}

void GroupPhase::fold_simt(int tsize, int side, int tm, const std::vector<FoldTask>& t) {
    std::vector<int> tiles(t.size());
    for (size_t i = 0; i < t.size(); ++i) tiles[i] = t[i].gx * t[i].gy * t[i].gz;
    int total = 0;
    const size_t off = put_tasks(t, tiles, &total);
    const size_t poff = ST_PREFIX_OF(off, FoldTask, t.size());
    const int nt = (int)t.size();
    if (total == 0) return;
    double bytes = 0.0, flops = 0.0;
    for (const FoldTask& k : t) {   // the algorithmic work of launch_gemm_fold, per task
        const double K0 = (k.n + 1) / 2, K1 = k.n / 2, batch = k.gz / 2;
        bytes += tsize * (K0 * K0 + K1 * K1 + 2.0 * k.other * k.n * batch);
        flops += 2.0 * k.other * (K0 * K0 + K1 * K1) * batch;
    }
    cudaStream_t s = s_;
    pend_.push_back({[=](const char* d) {
        const FoldTask* T = (const FoldTask*)(d + off);
        const int* P = (const int*)(d + poff);
        const int g = grid_for(total);
        // every tile shape sums the folded index in the same order with the same rounding, so the
        // shape does not change a result
        if (tsize == 4 && tm == 4) {
            if (side == 0)
                kg_fold<float, 4, 0><<<g, 256, 0, s>>>(T, P, nt);
            else
                kg_fold<float, 4, 1><<<g, 256, 0, s>>>(T, P, nt);
        } else if (tsize == 4) {
            if (side == 0)
                kg_fold<float, 2, 0><<<g, 256, 0, s>>>(T, P, nt);
            else
                kg_fold<float, 2, 1><<<g, 256, 0, s>>>(T, P, nt);
        } else {
            if (side == 0)
                kg_fold<double, 2, 0><<<g, 256, 0, s>>>(T, P, nt);
            else
                kg_fold<double, 2, 1><<<g, 256, 0, s>>>(T, P, nt);
        }
    }, tsize == 4 ? "g_fold32" : "g_fold64", bytes, flops});
}

void GroupPhase::fold_tc(int side, const std::vector<FoldTask>& t) {
    std::vector<int> tiles(t.size());
    for (size_t i = 0; i < t.size(); ++i) tiles[i] = t[i].gx * t[i].gy * t[i].gz;
    int total = 0;
    const size_t off = put_tasks(t, tiles, &total);
    const size_t poff = ST_PREFIX_OF(off, FoldTask, t.size());
    const int nt = (int)t.size();
    if (total == 0) return;
    double bytes = 0.0, flops = 0.0;
    for (const FoldTask& k : t) {
        const double K0 = (k.n + 1) / 2, K1 = k.n / 2, batch = k.gz / 2;
        bytes += 4.0 * (K0 * K0 + K1 * K1 + 2.0 * k.other * k.n * batch);
        flops += 2.0 * k.other * (K0 * K0 + K1 * K1) * batch;
    }
    cudaStream_t s = s_;
    pend_.push_back({[=](const char* d) {
        static const bool set = [] {
            cudaFuncSetAttribute(kg_fold_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, FTC_SMEM);
            cudaFuncSetAttribute(kg_fold_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, FTC_SMEM);
            return true;
        }();
        (void)set;
        const FoldTask* T = (const FoldTask*)(d + off);
        const int* P = (const int*)(d + poff);
        const int g = std::max(1, std::min(total, 152 * 3));   // up to three 66 KB CTAs an SM
        if (side == 0)
            kg_fold_tc<0><<<g, FTC_THREADS, FTC_SMEM, s>>>(T, P, nt);
        else
            kg_fold_tc<1><<<g, FTC_THREADS, FTC_SMEM, s>>>(T, P, nt);
    }, "g_fold_tc", bytes, flops});
}

void GroupPhase::stencil(int dim, const std::vector<StencilTask>& t) {
    if (t.empty()) return;
    std::vector<int> tiles(t.size());
    for (size_t i = 0; i < t.size(); ++i) tiles[i] = t[i].blocks * t[i].ncols;
    int total = 0;
    const size_t off = put_tasks(t, tiles, &total);
    const size_t poff = ST_PREFIX_OF(off, StencilTask, t.size());
    const int nt = (int)t.size();
    if (total == 0) return;
    double bytes = 0.0, flops = 0.0;
    for (const StencilTask& k : t) {   // each input read once, each output written once
        const double pts = (double)k.nx * k.ny * k.nz * k.ncols;
        const int nout = k.O2 ? 2 : 1;
        bytes += 8.0 * pts * (1 + nout + (k.beta != 0.0 ? 1 : 0));
        flops += 2.0 * (dim == 2 ? 9 : 27) * pts * nout;
    }
    cudaStream_t s = s_;
    pend_.push_back({[=](const char* d) {
        const StencilTask* T = (const StencilTask*)(d + off);
        const int* P = (const int*)(d + poff);
        if (dim == 2)
            kg_stencil<2><<<grid_for(total), dim3(32, 8), 0, s>>>(T, P, nt);
        else
            kg_stencil<3><<<grid_for(total), dim3(32, 8), 0, s>>>(T, P, nt);
    }, "g_stencil64", bytes, flops});
}

void GroupPhase::tn(bool df, const std::vector<TnTask>& t, bool hi) {
    hi = hi && df;
    if (t.empty()) return;
    const int cg = df ? TS_CG_DF : TS_CG;
    std::vector<int> tiles(t.size()), rtiles(t.size());
    int maxm = 1;
    size_t smem = 0;
    for (size_t i = 0; i < t.size(); ++i) {
        tiles[i] = t[i].nch * ((t[i].k + cg - 1) / cg);
        rtiles[i] = (t[i].k * t[i].m + 7) / 8;
        maxm = std::max(maxm, t[i].m);
        const size_t sm = df ? sizeof(float4) * (size_t)((t[i].m + 1) / 2) * t[i].rows
                             : sizeof(double) * (size_t)t[i].m * t[i].rows;
        smem = std::max(smem, sm);
    }
    int total = 0, rtotal = 0;
    const size_t off = put_tasks(t, tiles, &total);
    const size_t poff = ST_PREFIX_OF(off, TnTask, t.size());
    const size_t roff = put_tasks(t, rtiles, &rtotal);
    const size_t rpoff = ST_PREFIX_OF(roff, TnTask, t.size());
    const int nt = (int)t.size();
    double bytes = 0.0, flops = 0.0;
    for (const TnTask& k : t) {   // V and W read once, the chunk partials written and read once
        bytes += 8.0 * (double)k.n * (k.k + k.m) + 16.0 * (double)k.nch * k.k * k.m;
        flops += 2.0 * (double)k.n * k.k * k.m;
    }
    cudaStream_t s = s_;
    if (total > 0)
        pend_.push_back({[=](const char* d) {
            const TnTask* T = (const TnTask*)(d + off);
            const int* P = (const int*)(d + poff);
            with_maxm(maxm, [&](auto mm) {
                constexpr int MM = decltype(mm)::value;
                auto kern = hi ? kg_tn_partial<MM, true, true> : df ? kg_tn_partial<MM, true> : kg_tn_partial<MM, false>;
                static const bool set = [] {   // per instantiation: up to 64 KB of staged W
                    cudaFuncSetAttribute(kg_tn_partial<MM, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         8192 * 8);
                    cudaFuncSetAttribute(kg_tn_partial<MM, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         8192 * 8);
                    cudaFuncSetAttribute(kg_tn_partial<MM, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         8192 * 8);
                    return true;
                }();
                (void)set;
                kern<<<grid_for(total), TS_THREADS, smem, s>>>(T, P, nt);
            });
        }, hi ? "g_tn_hi" : df ? "g_tn_df" : "g_tn64", bytes, flops, rtotal == 0});
    if (rtotal > 0)
        pend_.push_back({[=](const char* d) {
            const TnTask* T = (const TnTask*)(d + roff);
            const int* P = (const int*)(d + rpoff);
            if (df)
                kg_tn_reduce<true><<<grid_for(rtotal), 256, 0, s>>>(T, P, nt);
            else
                kg_tn_reduce<false><<<grid_for(rtotal), 256, 0, s>>>(T, P, nt);
        }, total > 0 ? nullptr : (df ? "g_tn_df" : "g_tn64"), bytes, flops, true});
}

void GroupPhase::nn(bool df, const std::vector<NnTask>& t) {
    if (t.empty()) return;
    std::vector<int> tiles(t.size());
    int maxm = 1;
    for (size_t i = 0; i < t.size(); ++i) {
        tiles[i] = (t[i].n + 255) / 256;
        maxm = std::max(maxm, t[i].m);
    }
    int total = 0;
    const size_t off = put_tasks(t, tiles, &total);
    const size_t poff = ST_PREFIX_OF(off, NnTask, t.size());
    const int nt = (int)t.size();
    if (total == 0) return;
    double bytes = 0.0, flops = 0.0;
    for (const NnTask& k : t) {
        bytes += 8.0 * (double)k.n * (k.k + k.m * (k.beta == 0.0 ? 1 : 2));
        flops += 2.0 * (double)k.n * k.k * k.m;
    }
    cudaStream_t s = s_;
    pend_.push_back({[=](const char* d) {
        const NnTask* T = (const NnTask*)(d + off);
        const int* P = (const int*)(d + poff);
        with_maxm(maxm, [&](auto mm) {
            constexpr int MM = decltype(mm)::value;
            if (df)
                kg_nn<MM, true><<<grid_for(total), 256, 0, s>>>(T, P, nt);
            else
                kg_nn<MM, false><<<grid_for(total), 256, 0, s>>>(T, P, nt);
        });
    }, df ? "g_nn_df" : "g_nn64", bytes, flops});
}

void GroupPhase::trsm(const std::vector<TrsmTask>& t) {
    if (t.empty()) return;
    std::vector<int> tiles(t.size());
    for (size_t i = 0; i < t.size(); ++i) tiles[i] = (t[i].n + 256 * kSub - 1) / (256 * kSub);
    int total = 0;
    const size_t off = put_tasks(t, tiles, &total);
    const size_t poff = ST_PREFIX_OF(off, TrsmTask, t.size());
    const int nt = (int)t.size();
    if (total == 0) return;
    cudaStream_t s = s_;
    double bytes = 0.0, flops = 0.0;
    for (const TrsmTask& k : t) {
        bytes += 16.0 * (double)k.n * k.m;
        flops += (double)k.n * k.m * k.m;
    }
    pend_.push_back({[=](const char* d) {
        kg_trsm<<<grid_for(total), 256, 0, s>>>((const TrsmTask*)(d + off), (const int*)(d + poff), nt);
    }, "g_trsm", bytes, flops});
}

void GroupPhase::chol(const std::vector<CholTask>& t) {
    if (t.empty()) return;
    std::vector<int> tiles(t.size(), 1);
    int total = 0;
    const size_t off = put_tasks(t, tiles, &total);
    const size_t poff = ST_PREFIX_OF(off, CholTask, t.size());
    const int nt = (int)t.size();
    cudaStream_t s = s_;
    pend_.push_back({[=](const char* d) {
        kg_chol<<<grid_for(total), 32, 0, s>>>((const CholTask*)(d + off), (const int*)(d + poff), nt);
    }, "g_chol", 16.0 * 256 * t.size(), 0.0});
}

void GroupPhase::elem(const std::vector<ElemTask>& t) {
    if (t.empty()) return;
    std::vector<int> tiles(t.size());
    for (size_t i = 0; i < t.size(); ++i) tiles[i] = (int)(((long long)t[i].n * t[i].m + 256 * kSub - 1) / (256 * kSub));
    int total = 0;
    const size_t off = put_tasks(t, tiles, &total);
    const size_t poff = ST_PREFIX_OF(off, ElemTask, t.size());
    const int nt = (int)t.size();
    if (total == 0) return;
    double bytes = 0.0;
    for (const ElemTask& k : t) {   // bytes read and written per entry, by operation
        static const double per[5] = {16.0, 12.0, 12.0, 16.0, 16.0};
        bytes += (double)k.n * k.m * (per[k.op] + (k.b != 0.0 && (k.op == E_ADD32 || k.op == E_AXPBY) ? 8.0 : 0.0));
    }
    cudaStream_t s = s_;
    pend_.push_back({[=](const char* d) {
        kg_elem<<<grid_for(total), 256, 0, s>>>((const ElemTask*)(d + off), (const int*)(d + poff), nt);
    }, "g_elem", bytes, 0.0});
}

int GroupPhase::run() {
    if (pend_.empty()) {
        host_.clear();
        return ST_OK;
    }
    const size_t bytes = (host_.size() + 255) & ~size_t(255);
    ST_TRY(arena_->reserve(bytes, s_));
    char* hb = arena_->h + arena_->used;
    char* db = arena_->d + arena_->used;
    arena_->used += bytes;
    std::memcpy(hb, host_.data(), host_.size());
    ST_CUDA_TRY(cudaMemcpyAsync(db, hb, host_.size(), cudaMemcpyHostToDevice, s_));
    for (auto& p : pend_) {
        if (p.tag) st_prof_begin(s_, p.tag, p.bytes, p.flops);
        p.go(db);
        if (p.close) st_prof_end(s_);
        ST_LAUNCH_CHECK();
        ++launches_;
    }
    pend_.clear();
    host_.clear();
    return ST_OK;
}

}  // namespace stg
