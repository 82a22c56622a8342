// Device-side building blocks shared by the single-problem kernels
// (st_kernels.cu) and the grouped kernels of the batched solve
// (st_group.cu): the fast-diagonalisation epilogue, the tall-skinny and
// double-float product bodies, the box-stencil product, the block QR helpers
// and the elementwise column operations.  Each body computes one CTA's share
// of a launch from explicit block coordinates, so a single-problem kernel
// (coordinates from blockIdx) and a grouped kernel (coordinates of a tile of
// one instance of a batch) run the same arithmetic in the same order.
#pragma once

#include <cstdint>

#include "st_common.cuh"

namespace {

constexpr int kMaxCols = 16;   // widest block handled by the tall-skinny and SpMM kernels



__device__ __forceinline__ double fd_omega(const FdEpi& ep, long long e) {
    int x = (int)(e % ep.nx);
    long long t = e / ep.nx;
    int y = (int)(t % ep.ny);
    int z = (int)(t / ep.ny);
    double lam = ep.l0[x];
    double w = ep.c0[x];
    if (ep.dim > 1) {
        lam += ep.l1[y];
        w *= ep.c1[y];
    }
    if (ep.dim > 2) {
        lam += ep.l2[z];
        w *= ep.c2[z];
    }
    if (ep.kind == FD_MASS_INVERSE) return w;
    if (ep.kind == FD_RESOLVENT) return w / (ep.kappa * lam + ep.shift);
    return 1.0 / (ep.kappa * lam + ep.shift);
}

// The same weight in FP32 from the FP32 tables (no FP64 instruction).
__device__ __forceinline__ float fd_omega32(const FdEpi& ep, long long e) {
    int x = (int)(e % ep.nx);
    long long t = e / ep.nx;
    int y = (int)(t % ep.ny);
    int z = (int)(t / ep.ny);
    float lam = ep.f0[x];
    float w = ep.g0[x];
    if (ep.dim > 1) {
        lam += ep.f1[y];
        w *= ep.g1[y];
    }
    if (ep.dim > 2) {
        lam += ep.f2[z];
        w *= ep.g2[z];
    }
    const float kap = (float)ep.kappa, sh = (float)ep.shift;
    if (ep.kind == FD_MASS_INVERSE) return w;
    if (ep.kind == FD_RESOLVENT) return w / (kap * lam + sh);
    return 1.0f / (kap * lam + sh);
}


constexpr int TS_THREADS = 256;
constexpr int TS_CG = 16;      // basis columns per CTA of H = V^T W
constexpr int TS_CG_DF = 32;   // the same for the double-float product (half the restaging of W per basis column)
constexpr int TS_UNROLL = 8;   // independent loads in flight per lane
constexpr int TS_PIPE = 4;     // rows a lane per block of the software-pipelined double-float products

// Rows of one chunk of H = V^T W: enough chunks that chunks x column groups
// fill the GPU about four CTAs deep (a few basis columns need many short
// chunks to keep enough loads in flight), at least 128 rows, and a staged
// chunk of W of rows x m <= 8192 doubles.
__host__ __device__ inline int ts_rows(int n, int k, int m) {
    const int maxr = m <= 8 ? 1024 : 512;
    const long long groups = (k + 15) / 16;
    const long long want = 4 * 152;
    long long nch = (want + groups - 1) / groups;
    long long r = (n + nch - 1) / nch;
    r = ((r + 31) / 32) * 32;
    return (int)(r < 128 ? 128 : (r > maxr ? maxr : r));
}

// ---------------------------------------------------------------------------
// Double-float tall-skinny products.  FP64 runs at 1/64 of the FP32 rate on
// this chip, so the basis products of the mixed-precision solve use
// double-float arithmetic on the FP32 pipes instead (Dekker, "A floating-point
// technique for extending the available precision", 1971; Knuth, TAOCP
// vol. 2, 4.2.2, two-sum): a value is hi + lo with two floats, a product
// a*b = p + e with e = fma(a, b, -p) exact, and a running sum keeps its
// rounding error by two-sum.  Every 32 terms the pair is folded into an FP64
// accumulator.  The result carries about 48 significant bits, with no FP64
// instruction in the inner loops.  All FP32 operations are explicitly rounded
// intrinsics so that the compiler cannot contract them.  The basis is kept as
// (hi, lo) pairs (float2, 8 bytes per entry: the same traffic as FP64).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 df_split(double v) {
    float hi = __double2float_rn(v);
    float lo = __double2float_rn(v - (double)hi);
    return make_float2(hi, lo);
}

// (sh, sl) += (oh, ol) for two double-float partial sums (two-sum on the heads).
__device__ __forceinline__ void df_add(float& sh, float& sl, float oh, float ol) {
    float s = __fadd_rn(sh, oh);
    float z = __fsub_rn(s, sh);
    float t = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, z)), __fsub_rn(oh, z));
    sl = __fadd_rn(sl, __fadd_rn(t, ol));
    sh = s;
}

// Two double-float multiply-adds at once, (SH, SL)[c] += a * b_c for the two
// columns c of a pair, with the packed FP32 instructions of sm_100+ (each lane
// of a packed operation rounds exactly as the scalar one): the product
// p = a.hi b.hi with its exact error fma(a.hi, b.hi, -p) plus the two cross
// terms, then a two-sum of p onto the running head.
// b = (b0.hi, b1.hi, b0.lo, b1.lo).
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ void df_madd2(float2& SH, float2& SL, float2 a, float4 b) {
    const float2 Ax = make_float2(a.x, a.x), Ay = make_float2(a.y, a.y);
    const float2 Bx = make_float2(b.x, b.y), By = make_float2(b.z, b.w);
    const float2 P = __fmul2_rn(Ax, Bx);
    float2 E = __ffma2_rn(Ax, Bx, neg2(P));
    E = __ffma2_rn(Ax, By, E);
    E = __ffma2_rn(Ay, Bx, E);
    const float2 S = __fadd2_rn(SH, P);
    const float2 Z = __fadd2_rn(S, neg2(SH));
    const float2 T = __fadd2_rn(__fadd2_rn(SH, neg2(__fadd2_rn(S, neg2(Z)))), __fadd2_rn(P, neg2(Z)));
    SL = __fadd2_rn(SL, __fadd2_rn(T, E));
    SH = S;
}

// One step of a mode product's sum, rounded once (the same in every tile shape).
__device__ __forceinline__ float fold_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fold_fma(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename T, int TM, int SIDE>
__device__ __forceinline__ void fold_epilogue(T (&acc)[TM][TM], int M, int N, int m0, int n0, int tx, int ty,
                                              int par, T* __restrict__ C, long long ldc, const FdEpi& ep);

template <typename T, int TM, int SIDE>
__device__ __forceinline__ void gemm_fold_body(int n, int other, const T* __restrict__ X, long long ldx,
                                                   const T* __restrict__ H0, const T* __restrict__ H1,
                                                   const T* __restrict__ G0, const T* __restrict__ G1,
                                                   T* __restrict__ C, long long ldc, Batch2 bt, FdEpi ep, int bx, int by, int bz) {
    // FP32: the whole folded contraction of a 127-point direction (K <= 64) in one
    // staged step (fewer barriers, more loads in flight); FP64: 16 at a time
    constexpr int BM = 16 * TM, BN = 16 * TM, BK = sizeof(T) == 4 ? 64 : 16;
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BN];
    const int par = bz & 1;
    const int zb = bz >> 1;
    const int z1 = zb % bt.nb1, z2 = zb / bt.nb1;
    const int K = par ? n / 2 : (n + 1) / 2;   // folded length = outputs of this parity
    const int mid = (n & 1) ? (n - 1) / 2 : -1;
    const T sgn = par ? T(-1) : T(1);
    const int M = SIDE == 0 ? other : K;
    const int N = SIDE == 0 ? K : other;
    const int m0 = by * BM, n0 = bx * BN;
    if (m0 >= M || n0 >= N) return;   // the odd parity has one output fewer for odd n
    if (SIDE == 0) {
        X += (size_t)z1 * bt.sA1 + (size_t)z2 * bt.sA2;
    } else {
        X += (size_t)z1 * bt.sB1 + (size_t)z2 * bt.sB2;
    }
    C += (size_t)z1 * bt.sC1 + (size_t)z2 * bt.sC2;
    const T* Hp = par ? H1 : H0;   // K x K' (k-major), SIDE 0 right operand
    const T* Gp = par ? G1 : G0;   // K' x K (output-major), SIDE 1 left operand
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    T acc[TM][TM];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TM; ++j) acc[i][j] = T(0);
    for (int k0 = 0; k0 < K; k0 += BK) {
        for (int idx = tid; idx < BM * BK; idx += 256) {
            int mm = idx / BK, kk = idx % BK;
            int gm = m0 + mm, gk = k0 + kk;
            T v = T(0);
            if (gm < M && gk < K) {
                if (SIDE == 0) {
                    const T* row = X + (size_t)gm * ldx;
                    v = gk == mid ? row[gk] : row[gk] + sgn * row[n - 1 - gk];
                } else {
                    v = Gp[(size_t)gm * K + gk];
                }
            }
            As[kk][mm] = v;
        }
        for (int idx = tid; idx < BK * BN; idx += 256) {
            int kk = idx / BN, nn = idx % BN;
            int gk = k0 + kk, gn = n0 + nn;
            T v = T(0);
            if (gk < K && gn < N) {
                if (SIDE == 0) {
                    v = Hp[(size_t)gk * K + gn];
                } else {
                    v = gk == mid ? X[(size_t)gk * ldx + gn]
                                  : X[(size_t)gk * ldx + gn] + sgn * X[(size_t)(n - 1 - gk) * ldx + gn];
                }
            }
            Bs[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[TM], bb[TM];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < TM; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TM; ++j) acc[i][j] = fold_fma(a[i], bb[j], acc[i][j]);
        }
        __syncthreads();
    }
    fold_epilogue<T, TM, SIDE>(acc, M, N, m0, n0, tx, ty, par, C, ldc, ep);
}

// FP32 tile of 64 x 64 outputs, 4 x 4 a thread, with vector shared-memory reads: the staged operands sit
// in shared memory with the rows (columns) a thread owns -- ty, ty + 16, ty + 32, ty + 48 -- next to each
// other, so one 16-byte read feeds four outputs (two reads for sixteen FMAs, where the scalar 4 x 4 tile
// issues eight).  Every output is the same FMA chain over the folded index in the same order as in
// gemm_fold_body, so the two tiles give the same bits.  The folded index is staged 32 deep: eight entries
// of each operand a thread in registers between the loads and the shared stores, which leaves room for
// four CTAs an SM in the grouped kernel (64 deep held 128 registers and two CTAs; the load phases of a
// tile are then hidden by the other CTAs' FMAs).
template <int SIDE>
__device__ __forceinline__ void fold32_v4_body(int n, int other, const float* __restrict__ X, long long ldx,
                                               const float* __restrict__ H0, const float* __restrict__ H1,
                                               const float* __restrict__ G0, const float* __restrict__ G1,
                                               float* __restrict__ C, long long ldc, Batch2 bt, FdEpi ep, int bx,
                                               int by, int bz) {
    constexpr int BM = 64, BN = 64, BK = 32, LD = 68;   // row stride: 16-byte aligned, staging stores 4-way at most
    __shared__ __align__(16) float As[BK][LD];
    __shared__ __align__(16) float Bs[BK][LD];
    const int par = bz & 1;
    const int zb = bz >> 1;
    const int z1 = zb % bt.nb1, z2 = zb / bt.nb1;
    const int K = par ? n / 2 : (n + 1) / 2;
    const int mid = (n & 1) ? (n - 1) / 2 : -1;
    const float sgn = par ? -1.0f : 1.0f;
    const int M = SIDE == 0 ? other : K;
    const int N = SIDE == 0 ? K : other;
    const int m0 = by * BM, n0 = bx * BN;
    if (m0 >= M || n0 >= N) return;
    if (SIDE == 0) {
        X += (size_t)z1 * bt.sA1 + (size_t)z2 * bt.sA2;
    } else {
        X += (size_t)z1 * bt.sB1 + (size_t)z2 * bt.sB2;
    }
    C += (size_t)z1 * bt.sC1 + (size_t)z2 * bt.sC2;
    const float* Hp = par ? H1 : H0;
    const float* Gp = par ? G1 : G0;
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    auto pos = [](int r) { return (r & 15) * 4 + (r >> 4); };   // row r of the tile -> its staged slot
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
    constexpr int PER = BM * BK / 256;   // staged entries of each operand a thread
    for (int k0 = 0; k0 < K; k0 += BK) {
        // all loads of the chunk first (independent, in flight together), then the shared-memory stores
        float va[PER], vb[PER];
#pragma unroll
        for (int e = 0; e < PER; ++e) {
            const int idx = tid + 256 * e;
            const int mm = idx / BK, kk = idx % BK;
            const int gm = m0 + mm, gk = k0 + kk;
            float v = 0.0f;
            if (gm < M && gk < K) {
                if (SIDE == 0) {
                    const float* row = X + (size_t)gm * ldx;
                    v = gk == mid ? row[gk] : row[gk] + sgn * row[n - 1 - gk];
                } else {
                    v = Gp[(size_t)gm * K + gk];
                }
            }
            va[e] = v;
        }
#pragma unroll
        for (int e = 0; e < PER; ++e) {
            const int idx = tid + 256 * e;
            const int kk = idx / BN, nn = idx % BN;
            const int gk = k0 + kk, gn = n0 + nn;
            float v = 0.0f;
            if (gk < K && gn < N) {
                if (SIDE == 0) {
                    v = Hp[(size_t)gk * K + gn];
                } else {
                    v = gk == mid ? X[(size_t)gk * ldx + gn]
                                  : X[(size_t)gk * ldx + gn] + sgn * X[(size_t)(n - 1 - gk) * ldx + gn];
                }
            }
            vb[e] = v;
        }
#pragma unroll
        for (int e = 0; e < PER; ++e) {
            const int idx = tid + 256 * e;
            As[idx % BK][pos(idx / BK)] = va[e];
            Bs[idx / BN][pos(idx % BN)] = vb[e];
        }
        __syncthreads();
        const int kt = min(BK, K - k0);   // beyond it both operands are zero: the chain stops where K does
        for (int kk = 0; kk < kt; ++kk) {
            const float4 a = *reinterpret_cast<const float4*>(&As[kk][4 * ty]);
            const float4 b = *reinterpret_cast<const float4*>(&Bs[kk][4 * tx]);
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = __fmaf_rn(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
    fold_epilogue<float, 4, SIDE>(acc, M, N, m0, n0, tx, ty, par, C, ldc, ep);
}

template <typename T, int TM, int SIDE>
__device__ __forceinline__ void fold_epilogue(T (&acc)[TM][TM], int M, int N, int m0, int n0, int tx, int ty,
                                              int par, T* __restrict__ C, long long ldc, const FdEpi& ep) {
    const float fcoef = (float)ep.coef;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        int gm = m0 + ty + 16 * i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < TM; ++j) {
            int gn = n0 + tx + 16 * j;
            if (gn >= N) continue;
            // output coordinates of the unfolded product
            long long om = SIDE == 0 ? gm : 2LL * gm + par;
            long long on = SIDE == 0 ? 2LL * gn + par : gn;
            if constexpr (sizeof(T) == 4) {
                // FP32 epilogue: FP64 conversions and products here would run on the 1/64-rate pipe
                float f = fcoef;
                if (ep.scale) f *= fd_omega32(ep, ep.left ? om * ep.J + on : on);
                C[(size_t)om * ldc + on] = f * acc[i][j];
            } else {
                double f = ep.coef;
                if (ep.scale) {
                    long long e = ep.left ? om * ep.J + on : on;
                    f *= fd_omega(ep, e);
                }
                C[(size_t)om * ldc + on] = (T)(f * (double)acc[i][j]);
            }
        }
    }
}

// The mode product's tile body: the vector-read FP32 tile for 4 x 4 outputs a thread, else gemm_fold_body.
template <typename T, int TM, int SIDE>
__device__ __forceinline__ void fold_tile(int n, int other, const T* __restrict__ X, long long ldx,
                                          const T* __restrict__ H0, const T* __restrict__ H1,
                                          const T* __restrict__ G0, const T* __restrict__ G1, T* __restrict__ C,
                                          long long ldc, Batch2 bt, FdEpi ep, int bx, int by, int bz) {
    if constexpr (sizeof(T) == 4 && TM == 4)
        fold32_v4_body<SIDE>(n, other, X, ldx, H0, H1, G0, G1, C, ldc, bt, ep, bx, by, bz);
    else
        gemm_fold_body<T, TM, SIDE>(n, other, X, ldx, H0, H1, G0, G1, C, ldc, bt, ep, bx, by, bz);
}

template <typename T, int DIM, int YB, int ZB>
__device__ __forceinline__ void stencil_box_body(int nx, int ny, int nz, BoxPair<T> S, const T* __restrict__ X,
                                                     long long ldx, T beta, T* __restrict__ O1, long long ld1,
                                                     T* __restrict__ O2, long long ld2, int bx, int by) {
    constexpr int RY = YB + 2, RZ = DIM == 3 ? ZB + 2 : 1;
    constexpr int NV = RY * RZ * 3;
    const int nxs = (nx + 31) / 32, nyb = (ny + 8 * YB - 1) / (8 * YB);
    int b = bx;
    const int xs = b % nxs;
    b /= nxs;
    const int yb = b % nyb;
    const int zb = b / nyb;
    const int x = xs * 32 + threadIdx.x;
    const int y0 = (yb * 8 + threadIdx.y) * YB;
    const int z0 = zb * ZB;
    if (x >= nx || y0 >= ny || (DIM == 3 && z0 >= nz)) return;
    const long long nxy = (long long)nx * ny;
    const int c = by;
    const long long base = ((long long)(DIM == 3 ? z0 : 0) * ny + y0) * nx + x;
    const T* u = X + (size_t)c * ldx + base;
    T v[NV];
#pragma unroll
    for (int iz = 0; iz < RZ; ++iz)
#pragma unroll
        for (int iy = 0; iy < RY; ++iy)
#pragma unroll
            for (int ix = 0; ix < 3; ++ix) {
                const bool ok = x + ix - 1 >= 0 && x + ix - 1 < nx && y0 + iy - 1 >= 0 && y0 + iy - 1 < ny &&
                                (DIM < 3 || (z0 + iz - 1 >= 0 && z0 + iz - 1 < nz));
                const long long off = (long long)(DIM == 3 ? iz - 1 : 0) * nxy + (long long)(iy - 1) * nx + ix - 1;
                v[(iz * RY + iy) * 3 + ix] = ok ? u[off] : T(0);
            }
#pragma unroll
    for (int oz = 0; oz < (DIM == 3 ? ZB : 1); ++oz)
#pragma unroll
        for (int oy = 0; oy < YB; ++oy) {
            if (y0 + oy >= ny || (DIM == 3 && z0 + oz >= nz)) continue;
            T t1 = T(0), t2 = T(0);
#pragma unroll
            for (int e = 0; e < 27; ++e) {
                const int dz = e / 9 - 1, dy = (e / 3) % 3 - 1, dx = e % 3 - 1;
                if (DIM < 3 && dz != 0) continue;
                const T w = v[((DIM == 3 ? oz + 1 + dz : 0) * RY + oy + 1 + dy) * 3 + dx + 1];
                t1 += S.s[0][e] * w;
                if (O2) t2 += S.s[1][e] * w;
            }
            const long long at = base + (long long)(DIM == 3 ? oz : 0) * nxy + (long long)oy * nx;
            T* o1 = O1 + (size_t)c * ld1 + at;
            *o1 = beta == T(0) ? t1 : t1 + beta * *o1;
            if (O2) O2[(size_t)c * ld2 + at] = t2;
        }
}

template <int MAXM>
__device__ __forceinline__ void ts_tn_partial_body(int n, int k, int m, int rows,
                                                              const double* __restrict__ V, long long ldv,
                                                              const double* __restrict__ W, long long ldw,
                                                              double* __restrict__ part, double* Ws, int bx, int by) {
    const int chunk = bx;
    const int r0 = chunk * rows;
    const int nr = min(rows, n - r0);
    for (int idx = threadIdx.x; idx < m * rows; idx += TS_THREADS) {
        int b = idx / rows, rr = idx % rows;
        Ws[idx] = rr < nr ? W[(size_t)b * ldw + r0 + rr] : 0.0;
    }
    __syncthreads();
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    double* out = part + (size_t)chunk * k * m;
    for (int cc = warp; cc < TS_CG; cc += TS_THREADS / 32) {
        const int a = by * TS_CG + cc;
        if (a >= k) break;
        const double* v = V + (size_t)a * ldv + r0;
        double acc[MAXM];
#pragma unroll
        for (int b = 0; b < MAXM; ++b) acc[b] = 0.0;
        for (int base = lane; base < nr; base += 32 * TS_UNROLL) {
            double x[TS_UNROLL];
#pragma unroll
            for (int u = 0; u < TS_UNROLL; ++u) {
                int rr = base + 32 * u;
                x[u] = rr < nr ? v[rr] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < TS_UNROLL; ++u) {
                int rr = min(base + 32 * u, rows - 1);
#pragma unroll
                for (int b = 0; b < MAXM; ++b)
                    if (b < m) acc[b] += x[u] * Ws[b * rows + rr];
            }
        }
#pragma unroll
        for (int b = 0; b < MAXM; ++b) {
            if (b >= m) break;
            double t = acc[b];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
            if (lane == 0) out[(size_t)a * m + b] = t;
        }
    }
}

__device__ __forceinline__ void ts_reduce_body(int nchunks, int k, int m, const double* __restrict__ part, double* __restrict__ H,
                            long long ldh, int bx) {
    int idx = bx * (blockDim.x / 32) + threadIdx.x / 32;
    int lane = threadIdx.x % 32;
    if (idx >= k * m) return;
    double s = 0.0;
    for (int c = lane; c < nchunks; c += 32) s += part[(size_t)c * k * m + idx];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) {
        int a = idx / m, b = idx % m;
        H[(size_t)b * ldh + a] = s;
    }
}

template <int MAXM>
__device__ __forceinline__ void ts_nn_body(int n, int k, int m, double alpha, const double* __restrict__ V,
                                               long long ldv, const double* __restrict__ H, long long ldh,
                                               double beta, double* __restrict__ W, long long ldw, int bx) {
    constexpr int KT = 128;
    __shared__ double Hs[KT * MAXM];
    int r = bx * blockDim.x + threadIdx.x;
    double acc[MAXM];
#pragma unroll
    for (int b = 0; b < MAXM; ++b) acc[b] = 0.0;
    for (int a0 = 0; a0 < k; a0 += KT) {
        int kt = min(KT, k - a0);
        __syncthreads();
        for (int idx = threadIdx.x; idx < kt * m; idx += blockDim.x) {
            int a = idx / m, b = idx % m;
            Hs[a * MAXM + b] = H[(size_t)b * ldh + a0 + a];
        }
        __syncthreads();
        if (r < n) {
            for (int a = 0; a < kt; a += TS_UNROLL) {
                double x[TS_UNROLL];
#pragma unroll
                for (int u = 0; u < TS_UNROLL; ++u) x[u] = a + u < kt ? V[(size_t)(a0 + a + u) * ldv + r] : 0.0;
#pragma unroll
                for (int u = 0; u < TS_UNROLL; ++u) {
                    if (a + u >= kt) break;
#pragma unroll
                    for (int b = 0; b < MAXM; ++b)
                        if (b < m) acc[b] += x[u] * Hs[(a + u) * MAXM + b];
                }
            }
        }
    }
    if (r >= n) return;
#pragma unroll
    for (int b = 0; b < MAXM; ++b) {
        if (b >= m) break;
        double* w = W + (size_t)b * ldw + r;
        // explicit rounding: one product, then the other fused into the sum, so every kernel
        // that inlines this body rounds the same way
        *w = beta == 0.0 ? __dmul_rn(alpha, acc[b]) : __fma_rn(alpha, acc[b], __dmul_rn(beta, *w));
    }
}

__device__ __forceinline__ void to_df_body(int n, int m, const double* __restrict__ X, long long ldx, float2* __restrict__ Y,
                        long long ldy, int bx) {
    long long idx = bx * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)n * m) return;
    int j = (int)(idx / n), i = (int)(idx % n);
    Y[(size_t)j * ldy + i] = df_split(X[(size_t)j * ldx + i]);
}

// HI = true: the FP32 product of the leading parts only (V.hi^T W.hi, FP32 sums per lane, the lanes' sums
// combined by two-sum): the first pass of the mixed-precision block Gram-Schmidt, whose coefficients only
// need FP32 accuracy because the double-float second pass removes what the first one leaves.
template <int MAXM, bool HI = false>
__device__ __forceinline__ void ts_tn_df_partial_body(int n, int k, int m, int rows,
                                                                 const float2* __restrict__ V, long long ldv,
                                                                 const float2* __restrict__ W, long long ldw,
                                                                 float2* __restrict__ part, double* sm, int bx, int by) {
    constexpr int MP = (MAXM + 1) / 2;
    float4* Ws = reinterpret_cast<float4*>(sm);   // [pairs][rows]
    const int chunk = bx;
    const int r0 = chunk * rows;
    const int nr = min(rows, n - r0);
    const int np = (m + 1) / 2;
    for (int idx = threadIdx.x; idx < np * rows; idx += TS_THREADS) {
        const int q = idx / rows, rr = idx % rows;
        float2 w0 = make_float2(0.f, 0.f), w1 = make_float2(0.f, 0.f);
        if (rr < nr) {
            w0 = W[(size_t)(2 * q) * ldw + r0 + rr];
            if (2 * q + 1 < m) w1 = W[(size_t)(2 * q + 1) * ldw + r0 + rr];
        }
        Ws[idx] = make_float4(w0.x, w1.x, w0.y, w1.y);
    }
    __syncthreads();
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    float2* out = part + (size_t)chunk * k * m;
    // the FP32 product (HI) takes two basis columns a warp at a time (a0 and a0 + 8): twice the loads in
    // flight and one shared read of W for both, where its short FMA chains leave the loads exposed; the
    // double-float product keeps one (its longer chains already hide them, and a second set of
    // accumulators cost more in occupancy than it gave).  Each column's sum runs in the same order either way.
    constexpr int NW = TS_THREADS / 32, CPW = HI ? 2 : 1;
    for (int cc = warp; cc < TS_CG_DF; cc += CPW * NW) {
        const int a0 = by * TS_CG_DF + cc;
        if (a0 >= k) break;
        int na = 1;   // columns of this pass: a0, a0 + NW, ...
        while (na < CPW && cc + na * NW < TS_CG_DF && a0 + na * NW < k) ++na;
        const float2* v[CPW];
#pragma unroll
        for (int c = 0; c < CPW; ++c) v[c] = V + (size_t)(a0 + (c < na ? c : 0) * NW) * ldv + r0;
        float2 SH[CPW][MP], SL[CPW][MP];
#pragma unroll
        for (int c = 0; c < CPW; ++c)
#pragma unroll
            for (int q = 0; q < MP; ++q) SH[c][q] = SL[c][q] = make_float2(0.f, 0.f);
        // double-float: software-pipelined, the next block's V loads issued before this block's
        // multiply-adds, so they stay in flight through the dependent double-float chains; FP32 (short
        // chains): eight rows a lane loaded, then used.  The rows are taken in the same order either way.
        constexpr bool PIPE = !HI;
        constexpr int U = PIPE ? TS_PIPE : TS_UNROLL;
        float2 xv[CPW][U];
        auto load_block = [&](float2 (&x)[CPW][U], int b0) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int rr = b0 + 32 * u;
#pragma unroll
                for (int c = 0; c < CPW; ++c) x[c][u] = rr < nr && c < na ? v[c][rr] : make_float2(0.f, 0.f);
            }
        };
        if constexpr (PIPE) load_block(xv, lane);
        for (int base = lane; base < nr; base += 32 * U) {
            float2 xn[CPW][U];
            if constexpr (PIPE)
                load_block(xn, base + 32 * U);
            else
                load_block(xv, base);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                int rr = min(base + 32 * u, rows - 1);
#pragma unroll
                for (int q = 0; q < MP; ++q) {
                    if (q >= np) continue;
                    const float4 b = Ws[q * rows + rr];
#pragma unroll
                    for (int c = 0; c < CPW; ++c) {
                        if constexpr (HI)
                            SH[c][q] = __ffma2_rn(make_float2(xv[c][u].x, xv[c][u].x), make_float2(b.x, b.y), SH[c][q]);
                        else
                            df_madd2(SH[c][q], SL[c][q], xv[c][u], b);
                    }
                }
            }
            if constexpr (PIPE) {
#pragma unroll
                for (int u = 0; u < U; ++u)
#pragma unroll
                    for (int c = 0; c < CPW; ++c) xv[c][u] = xn[c][u];
            }
        }
#pragma unroll
        for (int c = 0; c < CPW; ++c) {
            if (c >= na) break;
            const int a = a0 + c * NW;
#pragma unroll
            for (int q = 0; q < MP; ++q) {
                if (q >= np) break;
#pragma unroll
                for (int h2 = 0; h2 < 2; ++h2) {
                    const int b = 2 * q + h2;
                    if (b >= m) break;
                    float h = h2 ? SH[c][q].y : SH[c][q].x, l = h2 ? SL[c][q].y : SL[c][q].x;
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) {
                        float oh = __shfl_xor_sync(0xffffffffu, h, off);
                        float ol = __shfl_xor_sync(0xffffffffu, l, off);
                        df_add(h, l, oh, ol);
                    }
                    if (lane == 0) out[(size_t)a * m + b] = make_float2(h, l);
                }
            }
        }
    }
}

__device__ __forceinline__ void ts_reduce_df_body(int nchunks, int k, int m, const float2* __restrict__ part, double* __restrict__ H,
                               long long ldh, int bx) {
    int idx = bx * (blockDim.x / 32) + threadIdx.x / 32;
    int lane = threadIdx.x % 32;
    if (idx >= k * m) return;
    double s = 0.0;
    for (int c = lane; c < nchunks; c += 32) {
        const float2 hl = part[(size_t)c * k * m + idx];
        s += (double)hl.x + (double)hl.y;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) {
        int a = idx / m, b = idx % m;
        H[(size_t)b * ldh + a] = s;
    }
}

template <int MAXM>
__device__ __forceinline__ void ts_nn_df_body(int n, int k, int m, double alpha, const float2* __restrict__ V,
                                                  long long ldv, const double* __restrict__ H, long long ldh,
                                                  double beta, double* __restrict__ W, long long ldw, int bx) {
    constexpr int KT = 128, MP = (MAXM + 1) / 2;
    __shared__ float4 Hs[KT * MP];
    const int np = (m + 1) / 2;
    int r = bx * blockDim.x + threadIdx.x;
    double acc[MAXM];
#pragma unroll
    for (int b = 0; b < MAXM; ++b) acc[b] = 0.0;
    for (int a0 = 0; a0 < k; a0 += KT) {
        int kt = min(KT, k - a0);
        __syncthreads();
        for (int idx = threadIdx.x; idx < kt * np; idx += blockDim.x) {
            const int a = idx / np, q = idx % np;
            const float2 h0 = df_split(H[(size_t)(2 * q) * ldh + a0 + a]);
            const float2 h1 = 2 * q + 1 < m ? df_split(H[(size_t)(2 * q + 1) * ldh + a0 + a]) : make_float2(0.f, 0.f);
            Hs[a * MP + q] = make_float4(h0.x, h1.x, h0.y, h1.y);
        }
        __syncthreads();
        if (r < n) {
            float2 SH[MP], SL[MP];
#pragma unroll
            for (int q = 0; q < MP; ++q) SH[q] = SL[q] = make_float2(0.f, 0.f);
            // software-pipelined like the product above: the next block's loads before this block's FMAs
            constexpr int U = TS_PIPE;
            float2 x[U];
            auto load_block = [&](float2 (&xb)[U], int b0) {
#pragma unroll
                for (int u = 0; u < U; ++u)
                    xb[u] = b0 + u < kt ? V[(size_t)(a0 + b0 + u) * ldv + r] : make_float2(0.f, 0.f);
            };
            load_block(x, 0);
            for (int a = 0; a < kt; a += U) {
                float2 xn[U];
                load_block(xn, a + U);
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (a + u >= kt) break;
#pragma unroll
                    for (int q = 0; q < MP; ++q)
                        if (q < np) df_madd2(SH[q], SL[q], x[u], Hs[(a + u) * MP + q]);
                }
#pragma unroll
                for (int u = 0; u < U; ++u) x[u] = xn[u];
            }
#pragma unroll
            for (int q = 0; q < MP; ++q) {
                if (2 * q < m) acc[2 * q] += (double)SH[q].x + (double)SL[q].x;
                if (2 * q + 1 < m && 2 * q + 1 < MAXM) acc[2 * q + 1] += (double)SH[q].y + (double)SL[q].y;
            }
        }
    }
    if (r >= n) return;
#pragma unroll
    for (int b = 0; b < MAXM; ++b) {
        if (b >= m) break;
        double* w = W + (size_t)b * ldw + r;
        // explicit rounding: one product, then the other fused into the sum, so every kernel
        // that inlines this body rounds the same way
        *w = beta == 0.0 ? __dmul_rn(alpha, acc[b]) : __fma_rn(alpha, acc[b], __dmul_rn(beta, *w));
    }
}

__device__ __forceinline__ void trsm_right_upper_body(int n, int m, const double* __restrict__ R, long long ldr, double* __restrict__ W,
                                   long long ldw, int bx) {
    __shared__ double Rs[kMaxCols * kMaxCols];
    for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) Rs[idx] = R[(size_t)(idx / m) * ldr + idx % m];
    __syncthreads();
    int r = bx * blockDim.x + threadIdx.x;
    if (r >= n) return;
    double x[kMaxCols];
#pragma unroll
    for (int j = 0; j < kMaxCols; ++j) x[j] = j < m ? W[(size_t)j * ldw + r] : 0.0;
#pragma unroll
    for (int j = 0; j < kMaxCols; ++j) {
        if (j >= m) break;
        double s = x[j];
#pragma unroll
        for (int i = 0; i < kMaxCols; ++i)
            if (i < j) s -= x[i] * Rs[j * m + i];   // R[i][j] stored column-major: Rs[j*m + i]
        x[j] = s / Rs[j * m + j];
    }
#pragma unroll
    for (int j = 0; j < kMaxCols; ++j)
        if (j < m) W[(size_t)j * ldw + r] = x[j];
}

__device__ __forceinline__ void chol_small_body(int m, const double* __restrict__ G, long long ldg, double* __restrict__ R,
                             long long ldr, double* __restrict__ flag) {
    __shared__ double a[kMaxCols][kMaxCols + 1];
    int t = threadIdx.x;
    for (int idx = t; idx < m * m; idx += 32) a[idx % m][idx / m] = G[(size_t)(idx / m) * ldg + idx % m];
    __syncwarp();
    bool bad = false;
    for (int j = 0; j < m; ++j) {
        double d = a[j][j];   // the same shared value in every lane: uniform branch
        if (!(d > 0.0)) {
            bad = true;
            break;
        }
        double rj = sqrt(d);
        __syncwarp();
        if (t > j && t < m) a[t][j] /= rj;
        if (t == j) a[j][j] = rj;
        __syncwarp();
        if (t > j && t < m) {
            double aij = a[t][j];
            for (int l = j + 1; l <= t; ++l) a[t][l] -= aij * a[l][j];
        }
        __syncwarp();
    }
    for (int idx = t; idx < m * m; idx += 32) {
        int i = idx % m, j = idx / m;   // R(i, j) = L(j, i) for i <= j
        double v = bad ? (i == j ? 1.0 : 0.0) : (i <= j ? a[j][i] : 0.0);
        R[(size_t)j * ldr + i] = v;
    }
    if (t == 0) *flag = bad ? 1.0 : 0.0;
}

template <typename S, typename D>
__device__ __forceinline__ void copy_cols_body(int n, int m, const S* __restrict__ X, long long ldx, D* __restrict__ Y, long long ldy,
                            double beta, int bx) {
    long long idx = bx * (long long)blockDim.x + threadIdx.x;
    long long tot = (long long)n * m;
    if (idx >= tot) return;
    int j = (int)(idx / n), i = (int)(idx % n);
    D v = (D)X[(size_t)j * ldx + i];
    D* y = Y + (size_t)j * ldy + i;
    if constexpr (sizeof(D) == 8)
        *y = beta == 0.0 ? v : (D)__fma_rn(beta, (double)(*y), (double)v);   // fused: the same in every kernel
    else
        *y = beta == 0.0 ? v : (D)__dmul_rn(beta, (double)(*y)) + v;
}

__device__ __forceinline__ void axpby_body(int n, int m, double a, const double* __restrict__ X, long long ldx, double b,
                        double* __restrict__ Y, long long ldy, int bx) {
    long long idx = bx * (long long)blockDim.x + threadIdx.x;
    long long tot = (long long)n * m;
    if (idx >= tot) return;
    int j = (int)(idx / n), i = (int)(idx % n);
    double* y = Y + (size_t)j * ldy + i;
    // explicit rounding (b y rounded, a x fused into the sum): the same in every kernel inlining this body
    *y = __fma_rn(a, X[(size_t)j * ldx + i], b == 0.0 ? 0.0 : __dmul_rn(b, *y));
}


// ---------------------------------------------------------------------------
// Folded mode product on the 5th-generation tensor cores (FP32 data, 3xTF32).
// The quantity of gemm_fold_body<float, TM, SIDE>: per parity p, the product
// of the folded operand with the half table (SIDE 0: C[line][2i'+p] =
// sum_k Xf[line][k] G_p[i'][k]; SIDE 1: C[2i'+p][col] = sum_k G_p[i'][k]
// Xf[k][col]) and the same epilogue.  A CTA of 256 threads computes a tile of
// 128 rows (the MMA's M) by FTC_N columns of D: it stages K in chunks of
// FTC_KC into shared memory as tf32 hi/lo planes (a = hi + lo, hi rounded to
// tf32) in the no-swizzle K-major core-matrix layout (8 rows x 16 bytes a core
// matrix), one thread issues D += Ahi Bhi + Ahi Blo + Alo Bhi with
// tcgen05.mma kind::tf32 (FP32 accumulator in TMEM; the dropped lo*lo term
// and tf32 rounding of the lo parts leave about FP32 accuracy), the CTA waits
// on an mbarrier (bounded), and the epilogue reads TMEM with tcgen05.ld,
// transposes through shared memory and stores coalesced.
// ---------------------------------------------------------------------------
constexpr int FTC_M = 128, FTC_N = 128, FTC_KC = 32, FTC_THREADS = 256;

// Built-in choice of the FP32 mode product's tile, the same for single and
// batched solves (so a problem's result does not depend on the path; in a
// batch of 2-column problems, grouping the tiles of many problems was measured
// no faster on the tensor cores, so the choice stays per problem): the tensor-core tile when
// the folded length fills the tile's 128 modes (FTC_MIN_K; at 64 modes, grids
// of 127 points a side, half of each MMA is padding and the SIMT tiles were
// faster in the 127^3 solve) and one launch has at least FTC_MIN_TILES of its
// 128 x 128 tiles, else the SIMT tiles.
constexpr int FTC_MIN_K = 128, FTC_MIN_TILES = 64;
__host__ __device__ inline bool fold_tc_default(int n, int other, int batch) {
    const int K0 = (n + 1) / 2;
    if (K0 < FTC_MIN_K) return false;
    // SIDE 0 tiles: lines x modes; SIDE 1: modes x lines -- the same count
    const long long tiles = (long long)((other + 127) / 128) * ((K0 + 127) / 128) * 2 * batch;
    return tiles >= FTC_MIN_TILES;
}
constexpr int FTC_PLANE = FTC_M * FTC_KC * 4;                  // 16 KB: one operand plane of a K chunk
constexpr int FTC_SMEM = 4 * FTC_PLANE > FTC_M * (FTC_N + 1) * 4 ? 4 * FTC_PLANE : FTC_M * (FTC_N + 1) * 4;
constexpr int FTC_TMEM_COLS = 128;
constexpr long long FTC_WAIT_LIMIT = 1ll << 24;                // mbarrier polls before giving up

__device__ __forceinline__ uint32_t ftc_smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: no swizzle, byte offsets between core matrices along K (lbo) and
// along M/N (sbo), descriptor version 1
__device__ __forceinline__ uint64_t ftc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

__device__ __forceinline__ float ftc_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// byte offset of (row, k) in a 128-row K-major plane of FTC_KC columns: core matrix (row/8, k/4) at
// ((k/4) * 16 + row/8) * 128
__device__ __forceinline__ int ftc_off(int row, int k) {
    return ((k >> 2) * 16 + (row >> 3)) * 128 + (row & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ void ftc_put(unsigned char* sm, int row, int k, float v) {
    const float hi = ftc_tf32(v);
    const int o = ftc_off(row, k);
    *(float*)(sm + o) = hi;                                   // plane 0: A hi (rows) / plane 2: B hi
    *(float*)(sm + FTC_PLANE + o) = ftc_tf32(v - hi);         // plane 1 / 3: lo
}

// TMEM allocation of the CTA (warp 0), done once per CTA.
__device__ __forceinline__ void ftc_alloc(uint32_t* slot) {
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(ftc_smem_u32(slot)),
                     "r"(FTC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
}
__device__ __forceinline__ void ftc_dealloc(uint32_t tmem) {
    if (threadIdx.x < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(FTC_TMEM_COLS));
}
__device__ __forceinline__ void ftc_mbar_init(uint64_t* mbar) {
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(ftc_smem_u32(mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
}

// Waits for the mbarrier's phase `ph`; false after FTC_WAIT_LIMIT polls.
__device__ __forceinline__ bool ftc_wait(uint64_t* mbar, uint32_t ph) {
    uint32_t done = 0;
    for (long long it = 0; it < FTC_WAIT_LIMIT && !done; ++it)
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done)
                     : "r"(ftc_smem_u32(mbar)), "r"(ph));
    return done != 0;
}

// One tile (bx, by, bz as gemm_fold_body with 128-row, FTC_N-column tiles).  Returns false if an MMA wait
// gave up (the tile's outputs are then NaN); *phase tracks the mbarrier's phase across calls.
template <int SIDE>
__device__ bool fold_tc_body(int n, int other, const float* __restrict__ X, long long ldx,
                             const float* __restrict__ G0, const float* __restrict__ G1, float* __restrict__ C,
                             long long ldc, Batch2 bt, const FdEpi& ep, int bx, int by, int bz, unsigned char* sm,
                             uint32_t tmem, uint64_t* mbar, uint32_t* phase) {
    const int par = bz & 1;
    const int zb = bz >> 1;
    const int z1 = zb % bt.nb1, z2 = zb / bt.nb1;
    const int K = par ? n / 2 : (n + 1) / 2;
    const int mid = (n & 1) ? (n - 1) / 2 : -1;
    const float sgn = par ? -1.f : 1.f;
    const int M = SIDE == 0 ? other : K;
    const int N = SIDE == 0 ? K : other;
    const int m0 = by * FTC_M, n0 = bx * FTC_N;
    if (m0 >= M || n0 >= N) return true;   // uniform over the CTA
    if (SIDE == 0)
        X += (size_t)z1 * bt.sA1 + (size_t)z2 * bt.sA2;
    else
        X += (size_t)z1 * bt.sB1 + (size_t)z2 * bt.sB2;
    C += (size_t)z1 * bt.sC1 + (size_t)z2 * bt.sC2;
    const float* Gp = par ? G1 : G0;   // K' x K, output-major: G_p[i'][k]
    const int tid = threadIdx.x;
    unsigned char* sa = sm;                       // A hi, A lo
    unsigned char* sb = sm + 2 * FTC_PLANE;       // B hi, B lo
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(FTC_N >> 3) << 17) |
                           ((uint32_t)(FTC_M >> 4) << 24);   // f32 accumulate, tf32 A and B, K-major, M 128
    const uint32_t kstride = (FTC_M / 8) * 128, mstride = 128;   // bytes between core matrices along K, M/N
    bool ok = true;
    for (int k0 = 0; k0 < K; k0 += FTC_KC) {
        // stage the chunk (zeros beyond the operands' edges)
        for (int idx = tid; idx < FTC_M * FTC_KC; idx += FTC_THREADS) {
            const int r = idx / FTC_KC, kk = idx % FTC_KC;
            const int gm = m0 + r, gk = k0 + kk;
            float v = 0.f;
            if (gm < M && gk < K) {
                if (SIDE == 0) {
                    const float* row = X + (size_t)gm * ldx;
                    v = gk == mid ? row[gk] : row[gk] + sgn * row[n - 1 - gk];
                } else {
                    v = Gp[(size_t)gm * K + gk];
                }
            }
            ftc_put(sa, r, kk, v);
        }
        for (int idx = tid; idx < FTC_N * FTC_KC; idx += FTC_THREADS) {
            int c, kk;
            if (SIDE == 0) {   // G_p rows: k contiguous
                c = idx / FTC_KC;
                kk = idx % FTC_KC;
            } else {           // X rows: columns contiguous
                kk = idx / FTC_N;
                c = idx % FTC_N;
            }
            const int gn = n0 + c, gk = k0 + kk;
            float v = 0.f;
            if (gn < N && gk < K) {
                if (SIDE == 0) {
                    v = Gp[(size_t)gn * K + gk];
                } else {
                    v = gk == mid ? X[(size_t)gk * ldx + gn]
                                  : X[(size_t)gk * ldx + gn] + sgn * X[(size_t)(n - 1 - gk) * ldx + gn];
                }
            }
            ftc_put(sb, c, kk, v);
        }
        asm volatile("fence.proxy.async.shared::cta;");   // generic-proxy stores visible to the tensor cores
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (tid == 0) {
            for (int s = 0; s < FTC_KC / 8; ++s) {
                const uint32_t ko = (uint32_t)s * 2 * kstride;
                const uint64_t ah = ftc_desc(ftc_smem_u32(sa) + ko, kstride, mstride);
                const uint64_t al = ftc_desc(ftc_smem_u32(sa + FTC_PLANE) + ko, kstride, mstride);
                const uint64_t bh = ftc_desc(ftc_smem_u32(sb) + ko, kstride, mstride);
                const uint64_t bl = ftc_desc(ftc_smem_u32(sb + FTC_PLANE) + ko, kstride, mstride);
                const uint64_t pa[3] = {ah, ah, al}, pb[3] = {bh, bl, bh};
#pragma unroll
                for (int t = 0; t < 3; ++t) {
                    const uint32_t acc = (k0 > 0 || s > 0 || t > 0) ? 1u : 0u;
                    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                 " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                                 "l"(pa[t]), "l"(pb[t]), "r"(idesc), "r"(acc));
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                ftc_smem_u32(mbar)));
        }
        if (!ftc_wait(mbar, *phase) && !ftc_wait(mbar, *phase)) ok = false;   // the chunk's MMAs are done
        *phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (!ok) break;
    }
    if (!ok) {
        // a wait gave up (no MMA completion after two bounded waits): the tile's outputs become NaN, so
        // the caller's solve stops on its non-finite checks, and the kernel takes no further tile
        for (int idx = tid; idx < FTC_M * FTC_N; idx += FTC_THREADS) {
            const int gm = m0 + idx / FTC_N, gn = n0 + idx % FTC_N;
            if (gm >= M || gn >= N) continue;
            const long long om = SIDE == 0 ? gm : 2LL * gm + par;
            const long long on = SIDE == 0 ? 2LL * gn + par : gn;
            C[(size_t)om * ldc + on] = __int_as_float(0x7fc00000);
        }
        return false;
    }
    // epilogue: warps w and w + 4 read TMEM lanes 32 (w % 4) .. +31 (rows), columns [0, 64) and [64, 128)
    const int warp = tid / 32, lane = tid % 32;
    float* T = reinterpret_cast<float*>(sm);   // 128 x (FTC_N + 1) transpose buffer over the operand planes
    const int row = 32 * (warp & 3) + lane;
    for (int c0 = (warp >> 2) * (FTC_N / 2); c0 < (warp >> 2) * (FTC_N / 2) + FTC_N / 2; c0 += 32) {
        uint32_t v[32];
        const uint32_t taddr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)c0;
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                     "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                     : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                       "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                       "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                       "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                       "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                     : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
        for (int j = 0; j < 32; ++j) T[row * (FTC_N + 1) + c0 + j] = __uint_as_float(v[j]);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    const float fcoef = (float)ep.coef;
    for (int idx = tid; idx < FTC_M * FTC_N; idx += FTC_THREADS) {
        const int r = idx / FTC_N, c = idx % FTC_N;   // a warp stores 32 consecutive columns of a row
        const int gm = m0 + r, gn = n0 + c;
        if (gm >= M || gn >= N) continue;
        const long long om = SIDE == 0 ? gm : 2LL * gm + par;
        const long long on = SIDE == 0 ? 2LL * gn + par : gn;
        float f = fcoef;
        if (ep.scale) f *= fd_omega32(ep, ep.left ? om * ep.J + on : on);
        C[(size_t)om * ldc + on] = f * T[r * (FTC_N + 1) + c];
    }
    __syncthreads();   // T is restaged by the next tile
    asm volatile("tcgen05.fence::after_thread_sync;");
    return true;
}

}  // namespace
