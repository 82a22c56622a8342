// Device kernels of the hot path: fused space-time apply, block SpMM,
// fast-diagonalisation mode products, tall-skinny block products.
#include <algorithm>
#include <cmath>

#include "st_common.cuh"
#include "st_dev.cuh"
#include "st_tune.h"

namespace {


// ---------------------------------------------------------------------------
// Fused space-time apply (Section 4, vec identity): column l of
// Y = M U D_t^T + A U C_t^T equals P u_l - N u_{l-1} with P = M + dt/2 A and
// N = M - dt/2 A on the shared CSR pattern.  One thread owns one row: its
// column indices and P, N values stay in registers while the thread walks a
// chunk of time columns, so the matrix is read once per chunk.  Lanes of a
// warp own consecutive rows, so the gathers U[col, l] of a warp are
// coalesced.  t_N of step l is carried to step l+1.
// ---------------------------------------------------------------------------
template <typename T, int MAXNNZ, int MINB = 1>
__global__ void __launch_bounds__(128, MINB) k_apply_reg(int n_h, int n_t, int chunk, const int* __restrict__ row_ptr,
                                                   const int* __restrict__ col, const T* __restrict__ pv,
                                                   const T* __restrict__ nv, const T* __restrict__ U, long long ldu,
                                                   T* __restrict__ Y, long long ldy) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_h) return;
    int l0 = blockIdx.y * chunk;
    int l1 = min(n_t, l0 + chunk);
    int a = row_ptr[r];
    int cnt = row_ptr[r + 1] - a;
    int c[MAXNNZ];
    T P[MAXNNZ], N[MAXNNZ];
#pragma unroll
    for (int e = 0; e < MAXNNZ; ++e) {
        bool ok = e < cnt;
        c[e] = ok ? col[a + e] : r;
        P[e] = ok ? pv[a + e] : T(0);
        N[e] = ok ? nv[a + e] : T(0);
    }
    T prevN = T(0);
    if (l0 > 0) {
        const T* u = U + (size_t)(l0 - 1) * ldu;
#pragma unroll
        for (int e = 0; e < MAXNNZ; ++e) prevN += N[e] * u[c[e]];
    }
    // STEPS time columns per pass: all their gathers are issued before the
    // FMAs, so a thread keeps STEPS x MAXNNZ loads in flight
    constexpr int STEPS = MAXNNZ <= 9 ? 4 : (sizeof(T) == 4 ? 2 : 1);
    int l = l0;
    for (; l + STEPS <= l1; l += STEPS) {
        T x[STEPS][MAXNNZ];
#pragma unroll
        for (int q = 0; q < STEPS; ++q) {
            const T* u = U + (size_t)(l + q) * ldu;
#pragma unroll
            for (int e = 0; e < MAXNNZ; ++e) x[q][e] = u[c[e]];
        }
#pragma unroll
        for (int q = 0; q < STEPS; ++q) {
            T tP = T(0), tN = T(0);
#pragma unroll
            for (int e = 0; e < MAXNNZ; ++e) {
                tP += P[e] * x[q][e];
                tN += N[e] * x[q][e];
            }
            Y[(size_t)(l + q) * ldy + r] = tP - prevN;
            prevN = tN;
        }
    }
    for (; l < l1; ++l) {
        const T* u = U + (size_t)l * ldu;
        T tP = T(0), tN = T(0);
#pragma unroll
        for (int e = 0; e < MAXNNZ; ++e) {
            T x = u[c[e]];
            tP += P[e] * x;
            tN += N[e] * x;
        }
        Y[(size_t)l * ldy + r] = tP - prevN;
        prevN = tN;
    }
}

// ---------------------------------------------------------------------------
// Fused space-time apply on a uniform box grid (2D, 3D): the same
// Y[:,l] = P u_l - N u_{l-1} without CSR gathers.  Every interior row of P and
// N carries the same 9 (27) stencil values, taken from the assembled CSR at
// set-up and passed as kernel parameters (constant bank, indexed at compile
// time), so the sums below equal the CSR kernel's term for term (a neighbour
// outside the box contributes an exact zero instead of a skipped entry).
// A thread owns one grid point and STEPS consecutive time columns (plus the
// column before them for N u_{l0-1}); all (STEPS+1) x 9 (27) loads are
// independent and issued together, with no shared memory and no barrier, so
// many CTAs per SM hide the latency.  Consecutive CTAs cover consecutive
// points of the same time chunk: the few U columns they touch stay in L2, so
// each U entry leaves HBM about once.
// ---------------------------------------------------------------------------
template <typename T>
struct BoxStencil {
    T p[27];
    T q[27];
};

// Register blocking: a thread owns YB x ZB grid points stacked in y (and z) at
// one x, so the (YB+2)(ZB+2) x 3 loads of a time column serve YB x ZB
// outputs (2D: 18 loads for 4 outputs instead of 36; 3D: 48 for 4 instead of
// 108).  A warp spans 32 consecutive x, so every load is coalesced.  The
// thread walks STEPS time columns, carrying N u_{l-1} per output, and loads
// the next column while it computes the current one.
template <typename T, int DIM, int YB, int ZB, int STEPS>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 && DIM == 2) ? 3 : 1) k_apply_box(int nx, int ny, int nz, int n_t, BoxStencil<T> S,
                                                   const T* __restrict__ U, long long ldu, T* __restrict__ Y,
                                                   long long ldy) {
    constexpr int RY = YB + 2, RZ = DIM == 3 ? ZB + 2 : 1;
    constexpr int NV = RY * RZ * 3;
    const int nxs = (nx + 31) / 32, nyb = (ny + 8 * YB - 1) / (8 * YB);
    int b = blockIdx.x;
    const int xs = b % nxs;
    b /= nxs;
    const int yb = b % nyb;
    const int zb = b / nyb;
    const int x = xs * 32 + threadIdx.x;
    const int y0 = (yb * 8 + threadIdx.y) * YB;
    const int z0 = zb * ZB;
    if (x >= nx || y0 >= ny || (DIM == 3 && z0 >= nz)) return;
    const long long nxy = (long long)nx * ny;
    const int l0 = blockIdx.y * STEPS;
    const int l1 = min(n_t, l0 + STEPS);
    const int c0 = l0 > 0 ? l0 - 1 : 0;
    // validity of the loaded rows and x neighbours
    bool okx[3], oky[RY], okz[RZ];
#pragma unroll
    for (int i = 0; i < 3; ++i) okx[i] = x + i - 1 >= 0 && x + i - 1 < nx;
#pragma unroll
    for (int i = 0; i < RY; ++i) oky[i] = y0 + i - 1 >= 0 && y0 + i - 1 < ny;
#pragma unroll
    for (int i = 0; i < RZ; ++i) okz[i] = DIM < 3 || (z0 + i - 1 >= 0 && z0 + i - 1 < nz);
    const long long base = ((long long)(DIM == 3 ? z0 : 0) * ny + y0) * nx + x;
    auto load = [&](int c, T* v) {
        const T* u = U + (size_t)c * ldu + base;
#pragma unroll
        for (int iz = 0; iz < RZ; ++iz)
#pragma unroll
            for (int iy = 0; iy < RY; ++iy)
#pragma unroll
                for (int ix = 0; ix < 3; ++ix) {
                    const bool ok = okx[ix] && oky[iy] && okz[iz];
                    const long long off = (long long)(DIM == 3 ? iz - 1 : 0) * nxy + (long long)(iy - 1) * nx + ix - 1;
                    v[(iz * RY + iy) * 3 + ix] = ok ? u[off] : T(0);
                }
    };
    // with prefetch (PF), column c+1 is loaded into the other buffer while c is computed
    constexpr bool PF = !(DIM == 3 && sizeof(T) == 8);   // FP64 3D: registers allow one buffer
    T va[NV], vb[PF ? NV : 1];
    T pn[YB * ZB];
#pragma unroll
    for (int o = 0; o < YB * ZB; ++o) pn[o] = T(0);
    if (PF) load(c0, va);
#pragma unroll 1
    for (int c = c0; c < l1; c += 2) {
        // column c in va; prefetch c + 1 into vb
        if (PF && c + 1 < l1) load(c + 1, vb);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int cc = c + h;
            if (cc >= l1) break;
            if (!PF) load(cc, va);
            const T* v = (h == 0 || !PF) ? va : vb;
            if (PF && h == 1 && cc + 1 < l1) load(cc + 1, va);   // the next pair's first column
#pragma unroll
            for (int oz = 0; oz < (DIM == 3 ? ZB : 1); ++oz)
#pragma unroll
                for (int oy = 0; oy < YB; ++oy) {
                    const int o = oz * YB + oy;
                    if (y0 + oy >= ny || (DIM == 3 && z0 + oz >= nz)) continue;
                    T tP = T(0), tN = T(0);
#pragma unroll
                    for (int e = 0; e < 27; ++e) {
                        const int dz = e / 9 - 1, dy = (e / 3) % 3 - 1, dx = e % 3 - 1;
                        if (DIM < 3 && dz != 0) continue;
                        const T w = v[((DIM == 3 ? oz + 1 + dz : 0) * RY + oy + 1 + dy) * 3 + dx + 1];
                        tP += S.p[e] * w;
                        tN += S.q[e] * w;
                    }
                    if (cc >= l0) Y[(size_t)cc * ldy + base + (long long)(DIM == 3 ? oz : 0) * nxy + (long long)oy * nx] =
                        tP - pn[o];
                    pn[o] = tN;
                }
        }
    }
}

// FP32 apply on a 2D box grid, two time columns a pass.  A lane holds U[x, c]
// and U[x, c + 1] of each of its YB + 2 rows as one f32x2 pair, so every term
// of the P and N stencils is one packed FMA for both columns; the sums run term
// for term in the order of k_apply_box (dy, dx lexicographic), so the results
// equal a column-at-a-time FP32 kernel's bit for bit.  x - 1 and x + 1 come
// from the neighbouring lanes by warp shuffles: a warp of 32 lanes yields 30
// outputs a row from one coalesced load a row and column (the two edge lanes
// only supply halo values).  A thread owns YB rows and walks NP pairs
// (c, c + 1), starting at c = l0 - 1 whose P u is not needed: Y_c = P u_c -
// N u_{c-1} with N u_{c-1} carried from the previous pair, and Y_{c+1} = P
// u_{c+1} - N u_c from the same pass.  Threads whose rows and columns are all in
// range load without predicates (only the CTAs at the grid's edges and the
// first and last time chunks take the checked loads).  Y is written with
// evict-first stores: nothing here reads it again.
template <int YB, int NP>
__global__ void __launch_bounds__(256, 2) k_apply_box_tp(int nx, int ny, int n_t, BoxStencil<float> S,
                                                         const float* __restrict__ U, long long ldu,
                                                         float* __restrict__ Y, long long ldy) {
    constexpr int RY = YB + 2;
    constexpr int STEPS = 2 * NP - 1;   // output columns a CTA
    const int nxs = (nx + 29) / 30;
    const int xs = blockIdx.x % nxs;
    const int yb = blockIdx.x / nxs;
    const int lane = threadIdx.x;
    const int x = xs * 30 + lane - 1;
    const int y0 = (yb * 8 + threadIdx.y) * YB;
    if (y0 >= ny) return;   // uniform over the warp: the shuffles see all lanes
    const bool okx = x >= 0 && x < nx;
    const bool emit = lane >= 1 && lane <= 30 && x < nx;
    bool ok[RY];
#pragma unroll
    for (int iy = 0; iy < RY; ++iy) ok[iy] = okx && y0 + iy - 1 >= 0 && y0 + iy - 1 < ny;
    const long long base = (long long)y0 * nx + x;
    const int l0 = blockIdx.y * STEPS;
    const bool inner = l0 >= 1 && l0 + STEPS <= n_t && okx && y0 >= 1 && y0 + YB < ny;
    float2 P2[9], N2[9];   // the 2D stencil: entries 9..17 of the 27-point tables (dz = 0)
#pragma unroll
    for (int e = 0; e < 9; ++e) {
        P2[e] = make_float2(S.p[9 + e], S.p[9 + e]);
        N2[e] = make_float2(S.q[9 + e], S.q[9 + e]);
    }
    const float* ub = U + base - nx;   // row y0 - 1
    // rows y0 - 1 .. y0 + YB of columns c0 and c0 + 1
    auto load = [&](int c0, float2* v) {
        const float* u0 = ub + (long long)c0 * ldu;
        const float* u1 = u0 + ldu;
        if (inner) {
#pragma unroll
            for (int iy = 0; iy < RY; ++iy) {
                v[iy].x = __ldg(u0 + iy * nx);
                v[iy].y = __ldg(u1 + iy * nx);
            }
        } else {
            const bool k0 = c0 >= 0 && c0 < n_t, k1 = c0 + 1 >= 0 && c0 + 1 < n_t;
#pragma unroll
            for (int iy = 0; iy < RY; ++iy) {
                v[iy].x = (k0 && ok[iy]) ? __ldg(u0 + iy * nx) : 0.f;
                v[iy].y = (k1 && ok[iy]) ? __ldg(u1 + iy * nx) : 0.f;
            }
        }
    };
    float2 buf[2][RY];
    float pn[YB];   // N u_{c0 - 1}
#pragma unroll
    for (int o = 0; o < YB; ++o) pn[o] = 0.f;
    load(l0 - 1, buf[0]);
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        const int c0 = l0 - 1 + 2 * j, c1 = c0 + 1;
        if (j + 1 < NP) load(c0 + 2, buf[(j + 1) % 2]);   // the next pair's loads in flight
        if (c0 >= n_t) break;
        const float2* v = buf[j % 2];
        float2 tP[YB], tN[YB];
#pragma unroll
        for (int o = 0; o < YB; ++o) tP[o] = tN[o] = make_float2(0.f, 0.f);
#pragma unroll
        for (int iy = 0; iy < RY; ++iy) {
            const float2 w0 = v[iy];
            float2 wm, wp;
            wm.x = __shfl_up_sync(0xffffffffu, w0.x, 1);
            wm.y = __shfl_up_sync(0xffffffffu, w0.y, 1);
            wp.x = __shfl_down_sync(0xffffffffu, w0.x, 1);
            wp.y = __shfl_down_sync(0xffffffffu, w0.y, 1);
#pragma unroll
            for (int oy = 0; oy < YB; ++oy) {
                const int dy = iy - 1 - oy;
                if (dy < -1 || dy > 1) continue;
                const int e = (dy + 1) * 3;
                tP[oy] = __ffma2_rn(P2[e], wm, tP[oy]);
                tN[oy] = __ffma2_rn(N2[e], wm, tN[oy]);
                tP[oy] = __ffma2_rn(P2[e + 1], w0, tP[oy]);
                tN[oy] = __ffma2_rn(N2[e + 1], w0, tN[oy]);
                tP[oy] = __ffma2_rn(P2[e + 2], wp, tP[oy]);
                tN[oy] = __ffma2_rn(N2[e + 2], wp, tN[oy]);
            }
        }
        if (emit) {
            float* yc = Y + (long long)c0 * ldy + base;
#pragma unroll
            for (int oy = 0; oy < YB; ++oy) {
                if (y0 + oy >= ny) continue;
                if (c0 >= l0) __stcs(yc + oy * nx, tP[oy].x - pn[oy]);
                if (c1 >= l0 && c1 < n_t) __stcs(yc + ldy + oy * nx, tP[oy].y - tN[oy].x);
            }
        }
#pragma unroll
        for (int o = 0; o < YB; ++o) pn[o] = tN[o].y;
    }
}

// ---------------------------------------------------------------------------
// Sum-factorised FP32 apply on a 3D box grid.  On a uniform box the Q1 mass
// and operator matrices are Kronecker products of 3-point 1D stencils,
// M = m_z (x) m_y (x) m_x and A = a_z (x) m_y (x) m_x + m_z (x) a_y (x) m_x +
// m_z (x) m_y (x) a_x (heat: a_d = kappa k_d; convection-diffusion:
// a_d = eps k_d + beta_d g_d), so with c = dt/2
//     P u = m_z S1 + c (m_z S2 + a_z S1),   N u = m_z S1 - c (m_z S2 + a_z S1),
//     S1 = (m_y (x) m_x) u,   S2 = (a_y (x) m_x + m_y (x) a_x) u:
// three passes of 3-point stencils (x, then y, then z) instead of the 27-point
// sums for P and N.  A warp spans 32 consecutive x and yields 30 outputs a row
// (the edge lanes supply halo values; x +- 1 by shuffles); a thread owns YB rows
// in y and walks ZB planes in z with a window of S1, S2 over three planes,
// the next plane's rows loaded while the current one is computed, then the
// next time column, carrying N u_{l-1} for its YB x ZB outputs.  Dirichlet
// neighbours are zeros at every stage, which is the tensor product of the
// interior 1D matrices.  Row pointers advance plane by plane (per-row 64-bit
// offsets hoisted out of the time loop would take the registers).
// ---------------------------------------------------------------------------
template <int YB, int ZB>
__global__ void __launch_bounds__(256, 2) k_apply_sf3(int nx, int ny, int nz, int n_t, int steps, SfStencil f,
                                                      const float* __restrict__ U, long long ldu, float* __restrict__ Y,
                                                      long long ldy) {
    const int nxs = (nx + 29) / 30, nyb = (ny + 8 * YB - 1) / (8 * YB);
    int b = blockIdx.x;
    const int xs = b % nxs;
    b /= nxs;
    const int yb = b % nyb;
    const int zb = b / nyb;
    const int lane = threadIdx.x;
    const int x = xs * 30 + lane - 1;
    const int y0 = (yb * 8 + threadIdx.y) * YB;
    const int z0 = zb * ZB;
    if (y0 >= ny) return;
    const bool okx = x >= 0 && x < nx;
    const bool emit = lane >= 1 && lane <= 30 && x < nx;
    bool oky[YB + 2];
#pragma unroll
    for (int r = 0; r < YB + 2; ++r) oky[r] = okx && y0 + r - 1 >= 0 && y0 + r - 1 < ny;
    const int l0 = blockIdx.y * steps;
    const int l1 = min(n_t, l0 + steps);
    float pn[ZB][YB];
#pragma unroll
    for (int j = 0; j < ZB; ++j)
#pragma unroll
        for (int o = 0; o < YB; ++o) pn[j][o] = 0.f;
    const long long nxy = (long long)nx * ny;
    // pointers advanced plane by plane (hoisted per-row 64-bit offsets would cost registers)
    const long long in0 = ((long long)(z0 - 1) * ny + (y0 - 1)) * nx + x;   // plane z0 - 1, row y0 - 1
    const long long out0 = ((long long)z0 * ny + y0) * nx + x;
#pragma unroll 1
    for (int c = l0 > 0 ? l0 - 1 : 0; c < l1; ++c) {
        const float* up = U + (long long)c * ldu + in0;
        float* yp = Y + (long long)c * ldy + out0;
        float s1a[YB], s2a[YB], s1b[YB], s2b[YB];
        float vv[2][YB + 2];
        {
            const bool okz = z0 - 1 >= 0;
#pragma unroll
            for (int r = 0; r < YB + 2; ++r) vv[0][r] = okz && oky[r] ? __ldg(up + r * nx) : 0.f;
        }
#pragma unroll
        for (int j = 0; j < ZB + 2; ++j) {
            if (j + 1 < ZB + 2) {   // plane j + 1 in flight while plane j is computed
                up += nxy;
                const int zn = z0 + j;
                const bool okz = zn < nz;
#pragma unroll
                for (int r = 0; r < YB + 2; ++r) vv[(j + 1) % 2][r] = okz && oky[r] ? __ldg(up + r * nx) : 0.f;
            }
            // keep the loads of later planes from being hoisted above this one (registers; a third plane in
            // flight was measured no faster)
            asm volatile("" ::: "memory");
            const int zz = z0 - 1 + j;
            float xm[YB + 2], xa[YB + 2];
#pragma unroll
            for (int r = 0; r < YB + 2; ++r) {
                const float v = vv[j % 2][r];
                const float wm = __shfl_up_sync(0xffffffffu, v, 1);
                const float wp = __shfl_down_sync(0xffffffffu, v, 1);
                xm[r] = fmaf(f.m1[0], wm + wp, f.m0[0] * v);
                xa[r] = fmaf(f.ap[0], wp, fmaf(f.am[0], wm, f.a0[0] * v));
            }
            float s1c[YB], s2c[YB];
#pragma unroll
            for (int o = 0; o < YB; ++o) {
                const int r = o + 1;
                s1c[o] = fmaf(f.m1[1], xm[r - 1] + xm[r + 1], f.m0[1] * xm[r]);
                const float yam = fmaf(f.ap[1], xm[r + 1], fmaf(f.am[1], xm[r - 1], f.a0[1] * xm[r]));
                const float yma = fmaf(f.m1[1], xa[r - 1] + xa[r + 1], f.m0[1] * xa[r]);
                s2c[o] = yam + yma;
            }
            if (j >= 2) {
                const int zo = zz - 1;
                if (zo < nz) {
#pragma unroll
                    for (int o = 0; o < YB; ++o) {
                        const float mz1 = fmaf(f.m1[2], s1a[o] + s1c[o], f.m0[2] * s1b[o]);
                        const float mz2 = fmaf(f.m1[2], s2a[o] + s2c[o], f.m0[2] * s2b[o]);
                        const float az1 = fmaf(f.ap[2], s1c[o], fmaf(f.am[2], s1a[o], f.a0[2] * s1b[o]));
                        const float t = mz2 + az1;
                        const float P = fmaf(f.hdt, t, mz1);
                        const float N = fmaf(-f.hdt, t, mz1);
                        if (c >= l0 && emit && y0 + o < ny) yp[o * nx] = P - pn[j - 2][o];
                        pn[j - 2][o] = N;
                    }
                }
                yp += nxy;
            }
#pragma unroll
            for (int o = 0; o < YB; ++o) {
                s1a[o] = s1b[o];
                s2a[o] = s2b[o];
                s1b[o] = s1c[o];
                s2b[o] = s2c[o];
            }
        }
    }
}

// Spatial products with a constant box stencil: O1[:,c] = S1 * X[:,c] (+ beta
// O1[:,c]) and, when O2 is given, O2[:,c] = S2 * X[:,c] from the same loads.
// Same thread layout and register blocking as the apply (a warp spans 32
// consecutive x; a thread owns YB x ZB points), one column per blockIdx.y.
// Only the vectors move: the stencil travels in the kernel parameters.

template <typename T, int DIM, int YB, int ZB>
__global__ void __launch_bounds__(256) k_stencil_box(int nx, int ny, int nz, BoxPair<T> S, const T* __restrict__ X,
                                                     long long ldx, T beta, T* __restrict__ O1, long long ld1,
                                                     T* __restrict__ O2, long long ld2) {
    stencil_box_body<T, DIM, YB, ZB>(nx, ny, nz, S, X, ldx, beta, O1, ld1, O2, ld2, blockIdx.x, blockIdx.y);
}

// FP32 variant of the constant-stencil product with the apply's shuffle scheme:
// a lane loads one x of each of its (YB+2)(ZB+2) rows and takes x +- 1 from its
// neighbours, a warp yields 30 outputs a row.  O = S * X (+ beta O).
template <int DIM, int YB, int ZB>
__global__ void __launch_bounds__(256) k_stencil_box_sh(int nx, int ny, int nz, BoxPair<float> S,
                                                        const float* __restrict__ X, long long ldx, float beta,
                                                        float* __restrict__ O, long long ldo) {
    constexpr int RY = YB + 2, RZ = DIM == 3 ? ZB + 2 : 1;
    const int nxs = (nx + 29) / 30, nyb = (ny + 8 * YB - 1) / (8 * YB);
    int b = blockIdx.x;
    const int xs = b % nxs;
    b /= nxs;
    const int yb = b % nyb;
    const int zb = b / nyb;
    const int lane = threadIdx.x;
    const int x = xs * 30 + lane - 1;
    const int y0 = (yb * 8 + threadIdx.y) * YB;
    const int z0 = zb * ZB;
    if (y0 >= ny || (DIM == 3 && z0 >= nz)) return;   // uniform over the warp
    const bool okx = x >= 0 && x < nx;
    const bool emit = lane >= 1 && lane <= 30 && x < nx;
    const long long nxy = (long long)nx * ny;
    const long long base = ((long long)(DIM == 3 ? z0 : 0) * ny + y0) * nx + x;
    const float* u = X + (size_t)blockIdx.y * ldx;
    float v[RY * RZ];
#pragma unroll
    for (int iz = 0; iz < RZ; ++iz)
#pragma unroll
        for (int iy = 0; iy < RY; ++iy) {
            const bool ok = okx && y0 + iy - 1 >= 0 && y0 + iy - 1 < ny &&
                            (DIM < 3 || (z0 + iz - 1 >= 0 && z0 + iz - 1 < nz));
            const long long off = (long long)(DIM == 3 ? iz - 1 : 0) * nxy + (long long)(iy - 1) * nx;
            v[iz * RY + iy] = ok ? __ldg(u + base + off) : 0.f;
        }
    float t[YB * ZB];
#pragma unroll
    for (int o = 0; o < YB * ZB; ++o) t[o] = 0.f;
#pragma unroll
    for (int iz = 0; iz < RZ; ++iz)
#pragma unroll
        for (int iy = 0; iy < RY; ++iy) {
            const float w0 = v[iz * RY + iy];
            const float wm = __shfl_up_sync(0xffffffffu, w0, 1);
            const float wp = __shfl_down_sync(0xffffffffu, w0, 1);
#pragma unroll
            for (int oz = 0; oz < (DIM == 3 ? ZB : 1); ++oz)
#pragma unroll
                for (int oy = 0; oy < YB; ++oy) {
                    const int dz = DIM == 3 ? iz - 1 - oz : 0, dy = iy - 1 - oy;
                    if (dz < -1 || dz > 1 || dy < -1 || dy > 1) continue;
                    const int e = (dz + 1) * 9 + (dy + 1) * 3;
                    const int o = oz * YB + oy;
                    t[o] += S.s[0][e] * wm;
                    t[o] += S.s[0][e + 1] * w0;
                    t[o] += S.s[0][e + 2] * wp;
                }
        }
    if (!emit) return;
    float* out = O + (size_t)blockIdx.y * ldo;
#pragma unroll
    for (int oz = 0; oz < (DIM == 3 ? ZB : 1); ++oz)
#pragma unroll
        for (int oy = 0; oy < YB; ++oy) {
            if (y0 + oy >= ny || (DIM == 3 && z0 + oz >= nz)) continue;
            const long long at = base + (long long)(DIM == 3 ? oz : 0) * nxy + (long long)oy * nx;
            const float r = t[oz * YB + oy];
            out[at] = beta == 0.f ? r : r + beta * out[at];
        }
}

// Generic CSR rows (any length): entries re-read from L1/L2 each step.
template <typename T>
__global__ void k_apply_generic(int n_h, int n_t, int chunk, const int* __restrict__ row_ptr,
                                const int* __restrict__ col, const T* __restrict__ pv, const T* __restrict__ nv,
                                const T* __restrict__ U, long long ldu, T* __restrict__ Y, long long ldy) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_h) return;
    int l0 = blockIdx.y * chunk;
    int l1 = min(n_t, l0 + chunk);
    int a = row_ptr[r], b = row_ptr[r + 1];
    T prevN = T(0);
    if (l0 > 0) {
        const T* u = U + (size_t)(l0 - 1) * ldu;
        for (int e = a; e < b; ++e) prevN += nv[e] * u[col[e]];
    }
    for (int l = l0; l < l1; ++l) {
        const T* u = U + (size_t)l * ldu;
        T tP = T(0), tN = T(0);
        for (int e = a; e < b; ++e) {
            T x = u[col[e]];
            tP += pv[e] * x;
            tN += nv[e] * x;
        }
        Y[(size_t)l * ldy + r] = tP - prevN;
        prevN = tN;
    }
}

// Block SpMM: OutM = M X, OutA = A X for ncols columns (K1b).
template <typename T, int MAXNNZ>
__global__ void __launch_bounds__(128) k_spmm_ma_reg(int n_h, int ncols, const int* __restrict__ row_ptr,
                                                     const int* __restrict__ col, const T* __restrict__ mv,
                                                     const T* __restrict__ av, const T* __restrict__ X, long long ldx,
                                                     T* __restrict__ OM, long long ldm, T* __restrict__ OA,
                                                     long long lda) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_h) return;
    int a0 = row_ptr[r];
    int cnt = row_ptr[r + 1] - a0;
    int c[MAXNNZ];
    T Mv[MAXNNZ], Av[MAXNNZ];
#pragma unroll
    for (int e = 0; e < MAXNNZ; ++e) {
        bool ok = e < cnt;
        c[e] = ok ? col[a0 + e] : r;
        Mv[e] = ok ? mv[a0 + e] : T(0);
        Av[e] = ok ? av[a0 + e] : T(0);
    }
    for (int j = 0; j < ncols; ++j) {
        const T* x = X + (size_t)j * ldx;
        T sm = T(0), sa = T(0);
#pragma unroll
        for (int e = 0; e < MAXNNZ; ++e) {
            T v = x[c[e]];
            sm += Mv[e] * v;
            sa += Av[e] * v;
        }
        if (OM) OM[(size_t)j * ldm + r] = sm;
        if (OA) OA[(size_t)j * lda + r] = sa;
    }
}

template <typename T>
__global__ void k_spmm_ma_generic(int n_h, int ncols, const int* __restrict__ row_ptr, const int* __restrict__ col,
                                  const T* __restrict__ mv, const T* __restrict__ av, const T* __restrict__ X,
                                  long long ldx, T* __restrict__ OM, long long ldm, T* __restrict__ OA,
                                  long long lda) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_h) return;
    int a0 = row_ptr[r], b0 = row_ptr[r + 1];
    for (int j = 0; j < ncols; ++j) {
        const T* x = X + (size_t)j * ldx;
        T sm = T(0), sa = T(0);
        for (int e = a0; e < b0; ++e) {
            T v = x[col[e]];
            sm += mv[e] * v;
            sa += av[e] * v;
        }
        if (OM) OM[(size_t)j * ldm + r] = sm;
        if (OA) OA[(size_t)j * lda + r] = sa;
    }
}

// Out = cm (M X) + ca (A X) + beta Out, FP64.
__global__ void k_spmm_comb64(int n_h, int ncols, const int* __restrict__ row_ptr, const int* __restrict__ col,
                              const double* __restrict__ mv, const double* __restrict__ av, double cm, double ca,
                              const double* __restrict__ X, long long ldx, double beta, double* __restrict__ O,
                              long long ldo) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_h) return;
    int a0 = row_ptr[r], b0 = row_ptr[r + 1];
    for (int j = 0; j < ncols; ++j) {
        const double* x = X + (size_t)j * ldx;
        double sm = 0.0, sa = 0.0;
        for (int e = a0; e < b0; ++e) {
            double v = x[col[e]];
            sm += mv[e] * v;
            sa += av[e] * v;
        }
        double o = cm * sm + ca * sa;
        double* po = O + (size_t)j * ldo + r;
        *po = beta == 0.0 ? o : o + beta * (*po);
    }
}

// CN right-hand side of step l: out = N u + sum_q F1[:,q] F2[l,q].
__global__ void k_cn_rhs(int n_h, const int* __restrict__ row_ptr, const int* __restrict__ col,
                         const double* __restrict__ nv, const double* __restrict__ u, const double* __restrict__ F1,
                         long long ldf1, const double* __restrict__ F2, long long ldf2, int l, int ncols,
                         double* __restrict__ out) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_h) return;
    double s = 0.0;
    if (u) {
        int a0 = row_ptr[r], b0 = row_ptr[r + 1];
        for (int e = a0; e < b0; ++e) s += nv[e] * u[col[e]];
    }
    for (int q = 0; q < ncols; ++q) s += F1[(size_t)q * ldf1 + r] * F2[(size_t)q * ldf2 + l];
    out[r] = s;
}

// ---------------------------------------------------------------------------
// Batched GEMM with row-major operands for the fast-diagonalisation mode
// products: C_b (M x N) = A_b (M x K) B_b (K x N), followed by an epilogue
// that scales by a constant and optionally by the spectral weight of the
// output entry.  64 x 64 tiles, 256 threads, 4 x 4 outputs per thread.
// ---------------------------------------------------------------------------

template <typename T, int TM>
__global__ void __launch_bounds__(256) k_gemm_rr(int M, int N, int K, const T* __restrict__ A, long long lda,
                                                 const T* __restrict__ B, long long ldb, T* __restrict__ C,
                                                 long long ldc, Batch2 bt, FdEpi ep) {
    constexpr int BM = 16 * TM, BN = 16 * TM, BK = 16;
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BN];
    int z = blockIdx.z;
    int z1 = z % bt.nb1, z2 = z / bt.nb1;
    A += (size_t)z1 * bt.sA1 + (size_t)z2 * bt.sA2;
    B += (size_t)z1 * bt.sB1 + (size_t)z2 * bt.sB2;
    C += (size_t)z1 * bt.sC1 + (size_t)z2 * bt.sC2;
    int tid = threadIdx.x;
    int tx = tid % 16, ty = tid / 16;
    int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    T acc[TM][TM];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TM; ++j) acc[i][j] = T(0);
    for (int k0 = 0; k0 < K; k0 += BK) {
        for (int idx = tid; idx < BM * BK; idx += 256) {
            int mm = idx / BK, kk = idx % BK;
            int gm = m0 + mm, gk = k0 + kk;
            As[kk][mm] = (gm < M && gk < K) ? A[(size_t)gm * lda + gk] : T(0);
        }
        for (int idx = tid; idx < BK * BN; idx += 256) {
            int kk = idx / BN, nn = idx % BN;
            int gk = k0 + kk, gn = n0 + nn;
            Bs[kk][nn] = (gk < K && gn < N) ? B[(size_t)gk * ldb + gn] : T(0);
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
                for (int j = 0; j < TM; ++j) acc[i][j] += a[i] * bb[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        int gm = m0 + ty + 16 * i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < TM; ++j) {
            int gn = n0 + tx + 16 * j;
            if (gn >= N) continue;
            double f = ep.coef;
            if (ep.scale) {
                long long e = ep.left ? (long long)gm * ep.J + gn : (long long)gn;
                f *= fd_omega(ep, e);
            }
            C[(size_t)gm * ldc + gn] = (T)(f * (double)acc[i][j]);
        }
    }
}

// ---------------------------------------------------------------------------
// Folded mode product.  The sine matrix Q[j][i] = sin((j+1)(i+1) pi/(n+1)) of
// the transforms satisfies Q[n-1-j][i] = (-1)^i Q[j][i], so an output of even
// index i needs only the folded input X[j] + X[n-1-j] and one of odd index only
// X[j] - X[n-1-j], for j below the middle (the middle entry of an odd n
// enters the even outputs alone: there Q is 0 for odd i).  Each product then
// becomes two half-size products (one per parity of the output index) with
// the tables H_p[k][i'] = Q[k][2i'+p] and G_p = H_p^T: half the FMAs of the
// full product.  blockIdx.z = 2 * batch + parity.
//   SIDE 0: C[line][i] = sum_j X[line][j] Q[j][i]   (the x direction)
//   SIDE 1: C[i][col]  = sum_j Q[i][j] X[j][col]    (the y and z directions)
// ---------------------------------------------------------------------------
template <typename T, int TM, int SIDE>
__global__ void __launch_bounds__(256) k_gemm_fold(int n, int other, const T* __restrict__ X, long long ldx,
                                                   const T* __restrict__ H0, const T* __restrict__ H1,
                                                   const T* __restrict__ G0, const T* __restrict__ G1,
                                                   T* __restrict__ C, long long ldc, Batch2 bt, FdEpi ep) {
    fold_tile<T, TM, SIDE>(n, other, X, ldx, H0, H1, G0, G1, C, ldc, bt, ep, blockIdx.x, blockIdx.y, blockIdx.z);
}

// The FP32 mode product on the tensor cores (one tile a CTA; see fold_tc_body).
template <int SIDE>
__global__ void __launch_bounds__(FTC_THREADS, 1) k_fold_tc(int n, int other, const float* __restrict__ X,
                                                           long long ldx, const float* __restrict__ G0,
                                                           const float* __restrict__ G1, float* __restrict__ C,
                                                           long long ldc, Batch2 bt, FdEpi ep) {
    extern __shared__ __align__(1024) unsigned char ftc_sm[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tslot;
    ftc_alloc(&tslot);
    ftc_mbar_init(&mbar);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    uint32_t ph = 0;
    fold_tc_body<SIDE>(n, other, X, ldx, G0, G1, C, ldc, bt, ep, blockIdx.x, blockIdx.y, blockIdx.z, ftc_sm, tslot,
                       &mbar, &ph);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    ftc_dealloc(tslot);
}

template <typename T, int SIDE>
int launch_gemm_fold(int n, int other, const T* X, long long ldx, const T* const* HG, T* C, long long ldc, int batch,
                     const Batch2& bt, const FdEpi& ep, cudaStream_t s, const char* tag) {
    if (n <= 0 || other <= 0 || batch <= 0) return ST_OK;
    const int K0 = (n + 1) / 2, K1 = n / 2;
    const int M = SIDE == 0 ? other : K0, N = SIDE == 0 ? K0 : other;
    // built-in tile choice: the tensor-core tile where fold_tc_default says so (FP32), else the SIMT tile
    // edge with the fewest tile rows per SM over both parities
    constexpr int kEdge[3] = {16, 32, 64};
    const bool tc_ok = sizeof(T) == 4;
    int def = 2;
    double best = 1e300;
    for (int c = 2; c >= 0; --c) {
        const int e = kEdge[c];
        long long tiles = (long long)((N + e - 1) / e) * ((M + e - 1) / e) * batch * 2;
        double eff = sizeof(T) == 8 ? 1.0 : (double)e / 64.0;
        double share = (double)((tiles + 151) / 152) * e * e / eff;
        if (share < 0.999 * best) {
            best = share;
            def = c;
        }
    }
    if (tc_ok && fold_tc_default(n, other, batch)) def = 3;
    auto fits = [&](int c) {
        if (c == 3) return tc_ok && (M + FTC_M - 1) / FTC_M <= 65535 && 2LL * batch <= 65535;
        const int e = kEdge[c];
        return (M + e - 1) / e <= 65535 && 2LL * batch <= 65535;
    };
    auto go = [&](int c) {
        if constexpr (sizeof(T) == 4) {
            if (c == 3) {
                static const bool set = [] {
                    cudaFuncSetAttribute(k_fold_tc<SIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize, FTC_SMEM);
                    return true;
                }();
                (void)set;
                dim3 grid((N + FTC_N - 1) / FTC_N, (M + FTC_M - 1) / FTC_M, 2 * batch);
                k_fold_tc<SIDE><<<grid, FTC_THREADS, FTC_SMEM, s>>>(n, other, X, ldx, HG[2], HG[3], C, ldc, bt, ep);
                return;
            }
        }
        const int e = kEdge[c];
        dim3 grid((N + e - 1) / e, (M + e - 1) / e, 2 * batch);
        if (e == 16)
            k_gemm_fold<T, 1, SIDE><<<grid, 256, 0, s>>>(n, other, X, ldx, HG[0], HG[1], HG[2], HG[3], C, ldc, bt, ep);
        else if (e == 32)
            k_gemm_fold<T, 2, SIDE><<<grid, 256, 0, s>>>(n, other, X, ldx, HG[0], HG[1], HG[2], HG[3], C, ldc, bt, ep);
        else
            k_gemm_fold<T, 4, SIDE><<<grid, 256, 0, s>>>(n, other, X, ldx, HG[0], HG[1], HG[2], HG[3], C, ldc, bt, ep);
    };
    const sttune::Key key{sttune::FOLD, (int)sizeof(T), SIDE, n, other, batch};
    int c = sttune::table().get(key);
    if (c < 0) {
        if (StTuneSession* ts = st_tune_session(s)) {
            // every variant writes all of C from X and the tables (no aliasing), so the
            // candidates may run on the launch's own operands
            bool valid[4] = {fits(0), fits(1), fits(2), fits(3)};
            double ms[4];
            ST_TRY(st_tune_measure(s, 4, valid, go, nullptr, ms));
            c = sttune::pick(ms, 4, def, 0.03);
            sttune::table().put(key, c);
            ++ts->tuned;
        }
    }
    if (c < 0 || !fits(c)) c = def;
    if (!fits(c)) return ST_EINVAL;
    double fma = (double)other * ((double)K0 * K0 + (double)K1 * K1) * batch;
    double bytes = (double)sizeof(T) * ((double)K0 * K0 + (double)K1 * K1 + 2.0 * (double)other * n * batch);
    st_prof_begin(s, tag, bytes, 2.0 * fma);
    go(c);
    st_prof_end(s);
    ST_LAUNCH_CHECK();
    return ST_OK;
}

template <typename T>
int launch_gemm_rr(int M, int N, int K, const T* A, long long lda, const T* B, long long ldb, T* C, long long ldc,
                   int batch, const Batch2& bt, const FdEpi& ep, cudaStream_t s, const char* tag) {
    if (M <= 0 || N <= 0 || batch <= 0) return ST_OK;
    // Tile edge 16, 32 or 64 (1, 2 or 4 outputs per thread and direction).
    // The busiest of the 152 SMs computes about ceil(tiles / 152) * edge^2
    // outputs.  FP64 FMAs are so slow on this chip (2 per clock per SM) that
    // this balance alone decides an FP64 product's time; in FP32 a small tile
    // also pays 2/TM shared loads per FMA, weighted in as 1/efficiency.  The
    // cheapest wins; ties go to the larger tile.
    int bm = 64;
    double best = 1e300;
    for (int e : {64, 32, 16}) {
        long long tiles = (long long)((N + e - 1) / e) * ((M + e - 1) / e) * batch;
        double eff = sizeof(T) == 8 ? 1.0 : (double)e / 64.0;
        double share = (double)((tiles + 151) / 152) * e * e / eff;
        if (share < 0.999 * best) {
            best = share;
            bm = e;
        }
    }
    dim3 grid((N + bm - 1) / bm, (M + bm - 1) / bm, batch);
    if (grid.y > 65535 || grid.z > 65535) return ST_EINVAL;
    double bytes = (double)sizeof(T) * ((double)M * K + ((double)K * N + (double)M * N) * batch);
    st_prof_begin(s, tag, bytes, 2.0 * M * N * (double)K * batch);
    if (bm == 16)
        k_gemm_rr<T, 1><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, bt, ep);
    else if (bm == 32)
        k_gemm_rr<T, 2><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, bt, ep);
    else
        k_gemm_rr<T, 4><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, bt, ep);
    st_prof_end(s);
    ST_LAUNCH_CHECK();
    return ST_OK;
}

// ---------------------------------------------------------------------------
// Tall-skinny products over the long dimension n (N_h).
// H = V^T W: each CTA reduces a chunk of rows into a k x m partial, a second
// kernel sums the partials in chunk order (deterministic).
// ---------------------------------------------------------------------------

// Partial products of H = V^T W over one chunk of rows and a group of TS_CG
// basis columns.  Each warp takes a column at a time; its lanes stride over
// the chunk's rows (coalesced loads of V, TS_UNROLL of them issued before the
// FMAs that use them) against the chunk of W in shared memory, then a fixed
// xor butterfly sums the lanes.  With 32+ rows per lane the butterfly's FP64
// adds are a small fraction of the FMAs (FP64 is the scarce unit).
template <int MAXM>
__global__ void __launch_bounds__(TS_THREADS) k_ts_tn_partial(int n, int k, int m, int rows,
                                                              const double* __restrict__ V, long long ldv,
                                                              const double* __restrict__ W, long long ldw,
                                                              double* __restrict__ part) {
    extern __shared__ double Ws[];
    ts_tn_partial_body<MAXM>(n, k, m, rows, V, ldv, W, ldw, part, Ws, blockIdx.x, blockIdx.y);
}

// One warp per output entry: lanes take every 32nd chunk, then a fixed
// butterfly sums the lanes, so the result does not depend on scheduling.
__global__ void k_ts_reduce(int nchunks, int k, int m, const double* __restrict__ part, double* __restrict__ H,
                            long long ldh) {
    ts_reduce_body(nchunks, k, m, part, H, ldh, blockIdx.x);
}

// W = beta W + alpha V H, one thread per row, H staged through shared memory;
// TS_UNROLL basis entries of the row are loaded before the FMAs that use them.
template <int MAXM>
__global__ void __launch_bounds__(256) k_ts_nn(int n, int k, int m, double alpha, const double* __restrict__ V,
                                               long long ldv, const double* __restrict__ H, long long ldh,
                                               double beta, double* __restrict__ W, long long ldw) {
    ts_nn_body<MAXM>(n, k, m, alpha, V, ldv, H, ldh, beta, W, ldw, blockIdx.x);
}


// Partial H = V^T W as k_ts_tn_partial, with V and W both in double-float
// (W split once by the caller, not once per CTA: the split costs FP64).  W's
// chunk is staged as column pairs (hi, hi, lo, lo) so that one 16-byte shared
// load feeds a packed df_madd2 for two columns.  The lanes' partial sums are
// combined by a double-float butterfly and stored as (hi, lo) float pairs: no
// FP64 instruction runs here (FP64 is 1/64 of FP32); k_ts_reduce_df folds
// them.
__global__ void k_to_df(int n, int m, const double* __restrict__ X, long long ldx, float2* __restrict__ Y,
                        long long ldy) {
    to_df_body(n, m, X, ldx, Y, ldy, blockIdx.x);
}

template <int MAXM, bool HI>
__global__ void __launch_bounds__(TS_THREADS) k_ts_tn_df_partial(int n, int k, int m, int rows,
                                                                 const float2* __restrict__ V, long long ldv,
                                                                 const float2* __restrict__ W, long long ldw,
                                                                 float2* __restrict__ part) {
    extern __shared__ double sm[];
    ts_tn_df_partial_body<MAXM, HI>(n, k, m, rows, V, ldv, W, ldw, part, sm, blockIdx.x, blockIdx.y);
}

// H = sum over chunks of the (hi, lo) partials, each folded to FP64 first:
// a warp per output, fixed order (as k_ts_reduce).
__global__ void k_ts_reduce_df(int nchunks, int k, int m, const float2* __restrict__ part, double* __restrict__ H,
                               long long ldh) {
    ts_reduce_df_body(nchunks, k, m, part, H, ldh, blockIdx.x);
}

// W = beta W + alpha V H with V in double-float, one thread per row; H is
// split once per CTA into shared memory as column pairs (hi, hi, lo, lo), the
// double-float sums run two columns at a time (df_madd2) and are folded into
// FP64 every 128 basis columns.
template <int MAXM>
__global__ void __launch_bounds__(256) k_ts_nn_df(int n, int k, int m, double alpha, const float2* __restrict__ V,
                                                  long long ldv, const double* __restrict__ H, long long ldh,
                                                  double beta, double* __restrict__ W, long long ldw) {
    ts_nn_df_body<MAXM>(n, k, m, alpha, V, ldv, H, ldh, beta, W, ldw, blockIdx.x);
}

__global__ void k_trsm_right_upper(int n, int m, const double* __restrict__ R, long long ldr, double* __restrict__ W,
                                   long long ldw) {
    trsm_right_upper_body(n, m, R, ldr, W, ldw, blockIdx.x);
}

// Cholesky factor of a small SPD matrix by one warp, lane i owning row i of
// the lower factor L (R = L^T): column j is scaled by its pivot, then each
// lane updates its row of the trailing block.
__global__ void k_chol_small(int m, const double* __restrict__ G, long long ldg, double* __restrict__ R,
                             long long ldr, double* __restrict__ flag) {
    chol_small_body(m, G, ldg, R, ldr, flag);
}

template <typename S, typename D>
__global__ void k_copy_cols(int n, int m, const S* __restrict__ X, long long ldx, D* __restrict__ Y, long long ldy,
                            double beta) {
    copy_cols_body<S, D>(n, m, X, ldx, Y, ldy, beta, blockIdx.x);
}

__global__ void k_axpby(int n, int m, double a, const double* __restrict__ X, long long ldx, double b,
                        double* __restrict__ Y, long long ldy) {
    axpby_body(n, m, a, X, ldx, b, Y, ldy, blockIdx.x);
}

// ---------------------------------------------------------------------------
// Batched flexible GMRES: m independent Arnoldi processes, one per column of a
// block, advanced together.  The Krylov blocks are interleaved: vector i of
// column c is Z + (i m + c) n.  Each kernel covers all m columns, so a step
// costs the same launches for any m and no column's coefficients leave the
// device until the host checks convergence.
// ---------------------------------------------------------------------------

// part[(chunk m + c) kk + i] = sum over the chunk's rows of Z_i[:,c] . Z_{kk-1}[:,c]
// for i < kk: the last vector is the one being orthogonalised, so i = kk - 1
// is its squared norm.  The chunk of that vector is staged in shared memory;
// a warp per basis vector, lanes over rows, a fixed butterfly.
// T = double, or float for the inner solve of iterative refinement: FP32
// products summed per lane in FP32 (a few dozen terms), combined in FP64.
template <typename T>
__global__ void __launch_bounds__(256) k_gm_dot_partial(int n, int kk, int m, int rows, const T* __restrict__ Z,
                                                        double* __restrict__ part) {
    extern __shared__ double us_raw[];
    T* us = reinterpret_cast<T*>(us_raw);
    const int c = blockIdx.y;
    const long long r0 = (long long)blockIdx.x * rows;
    const int rn = (int)min((long long)rows, (long long)n - r0);
    const T* u = Z + ((size_t)(kk - 1) * m + c) * n + r0;
    for (int t = threadIdx.x; t < rn; t += blockDim.x) us[t] = u[t];
    __syncthreads();
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    for (int i = warp; i < kk; i += blockDim.x / 32) {
        const T* z = Z + ((size_t)i * m + c) * n + r0;
        T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
        int t = lane;
        for (; t + 96 < rn; t += 128) {
            s0 += z[t] * us[t];
            s1 += z[t + 32] * us[t + 32];
            s2 += z[t + 64] * us[t + 64];
            s3 += z[t + 96] * us[t + 96];
        }
        for (; t < rn; t += 32) s0 += z[t] * us[t];
        // the lanes combine in T (FP64 adds on FP32 data would run on the 1/64-rate pipe);
        // the chunk partials are summed in FP64 by k_gm_reduce
        T sum = (s0 + s1) + (s2 + s3);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
        if (lane == 0) part[((size_t)blockIdx.x * m + c) * kk + i] = (double)sum;
    }
}

// H[c ldh + i] = sum over chunks of part: a warp per (c, i), fixed order.
__global__ void k_gm_reduce(int nch, int kk, int m, const double* __restrict__ part, double* __restrict__ H, int ldh) {
    const int idx = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x % 32;
    if (idx >= kk * m) return;
    const int c = idx / kk, i = idx % kk;
    double s = 0.0;
    for (int ch = lane; ch < nch; ch += 32) s += part[((size_t)ch * m + c) * kk + i];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) H[(size_t)c * ldh + i] = s;
}

// Z_nb[:,c] -= sum_{i < nb} Z_i[:,c] H[c ldh + i], a thread per row for all m
// columns.  With H1 (the first pass's coefficients) the step ends here: H holds
// the second pass's coefficients and, at i = nb, the squared norm of the vector
// before this update, so the new norm is h = sqrt(H[nb] - sum H[i]^2); the
// vector is divided by h (set to zero when h = 0) and CTA 0 writes column jcol
// of each column's Hessenberg matrix, Hd[c ldhd + jcol (J + 1) + i] =
// H1[i] + H[i] (i < nb) and h (i = nb).
template <typename T, int MAXM>
__global__ void __launch_bounds__(256) k_gm_update(int n, int nb, int m, T* __restrict__ Z,
                                                   const double* __restrict__ H, int ldh,
                                                   const double* __restrict__ H1, int ldh1, double* __restrict__ Hd,
                                                   long long ldhd, int jcol, int J) {
    extern __shared__ double hs[];   // m x (nb + 1) coefficients, then m scale factors, then the coefficients in T
    double* inv = hs + (size_t)m * (nb + 1);
    T* ht = reinterpret_cast<T*>(inv + m);
    for (int t = threadIdx.x; t < m * (nb + 1); t += blockDim.x) hs[t] = H[(size_t)(t / (nb + 1)) * ldh + t % (nb + 1)];
    __syncthreads();
    if (H1 && threadIdx.x < m) {
        const int c = threadIdx.x;
        double ss = 0.0;
        for (int i = 0; i < nb; ++i) ss += hs[c * (nb + 1) + i] * hs[c * (nb + 1) + i];
        const double nu2 = hs[c * (nb + 1) + nb] - ss;
        const double h = nu2 > 0.0 ? sqrt(nu2) : 0.0;
        inv[c] = h > 0.0 ? 1.0 / h : 0.0;
        if (blockIdx.x == 0) {
            double* col = Hd + (size_t)c * ldhd + (size_t)jcol * (J + 1);
            for (int i = 0; i < nb; ++i) col[i] = H1[(size_t)c * ldh1 + i] + hs[c * (nb + 1) + i];
            col[nb] = h;
        }
    }
    for (int t = threadIdx.x; t < m * (nb + 1); t += blockDim.x) ht[t] = (T)hs[t];
    __syncthreads();
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    T invt[MAXM];
#pragma unroll
    for (int c = 0; c < MAXM; ++c) invt[c] = (H1 && c < m) ? (T)inv[c] : T(1);
    T acc[MAXM];
#pragma unroll
    for (int c = 0; c < MAXM; ++c) acc[c] = c < m ? Z[((size_t)nb * m + c) * n + r] : T(0);
    for (int i = 0; i < nb; ++i) {
        T z[MAXM];
#pragma unroll
        for (int c = 0; c < MAXM; ++c) z[c] = c < m ? Z[((size_t)i * m + c) * n + r] : T(0);
#pragma unroll
        for (int c = 0; c < MAXM; ++c)
            if (c < m) acc[c] -= z[c] * ht[c * (nb + 1) + i];   // ht holds m columns only
    }
#pragma unroll
    for (int c = 0; c < MAXM; ++c)
        if (c < m) Z[((size_t)nb * m + c) * n + r] = H1 ? acc[c] * invt[c] : acc[c];
}

// The first pass's update fused with the second pass's dot products, one CTA
// per chunk of rows (the chunks of k_gm_dot_partial): the chunk's new vector
// U = Z_nb - sum_i Z_i h1_i is written to Z and kept in shared memory, then the
// partial dots Z_i . U (i < nb) and U . U are taken while the chunk's Z_i are
// still in L2, so the second pass reads the basis from L2 instead of HBM.
template <typename T, int MAXM>
__global__ void __launch_bounds__(256) k_gm_update_dot(int n, int nb, int m, int rows, T* __restrict__ Z,
                                                       const double* __restrict__ H, int ldh,
                                                       double* __restrict__ part) {
    extern __shared__ double sm_ud[];
    double* hs = sm_ud;                                   // m x (nb + 1) first-pass coefficients
    T* ht = reinterpret_cast<T*>(hs + (size_t)m * (nb + 1));
    T* us = ht + (size_t)m * (nb + 1);                    // [m][rows] the chunk's new vectors
    for (int t = threadIdx.x; t < m * (nb + 1); t += blockDim.x) {
        hs[t] = H[(size_t)(t / (nb + 1)) * ldh + t % (nb + 1)];
        ht[t] = (T)hs[t];
    }
    __syncthreads();
    const long long r0 = (long long)blockIdx.x * rows;
    const int rn = (int)min((long long)rows, (long long)n - r0);
    for (int t = threadIdx.x; t < rn; t += blockDim.x) {
        const long long r = r0 + t;
        T acc[MAXM];
#pragma unroll
        for (int c = 0; c < MAXM; ++c) acc[c] = c < m ? Z[((size_t)nb * m + c) * n + r] : T(0);
        for (int i = 0; i < nb; ++i) {
            T z[MAXM];
#pragma unroll
            for (int c = 0; c < MAXM; ++c) z[c] = c < m ? Z[((size_t)i * m + c) * n + r] : T(0);
#pragma unroll
            for (int c = 0; c < MAXM; ++c)
                if (c < m) acc[c] -= z[c] * ht[c * (nb + 1) + i];
        }
#pragma unroll
        for (int c = 0; c < MAXM; ++c)
            if (c < m) {
                Z[((size_t)nb * m + c) * n + r] = acc[c];
                us[(size_t)c * rows + t] = acc[c];
            }
    }
    __syncthreads();
    const int kk = nb + 1;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    for (int q = warp; q < m * kk; q += blockDim.x / 32) {
        const int c = q / kk, i = q % kk;
        const T* u = us + (size_t)c * rows;
        const T* z = i < nb ? Z + ((size_t)i * m + c) * n + r0 : u;
        T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
        int t = lane;
        for (; t + 96 < rn; t += 128) {
            s0 += z[t] * u[t];
            s1 += z[t + 32] * u[t + 32];
            s2 += z[t + 64] * u[t + 64];
            s3 += z[t + 96] * u[t + 96];
        }
        for (; t < rn; t += 32) s0 += z[t] * u[t];
        T sum = (s0 + s1) + (s2 + s3);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
        if (lane == 0) part[((size_t)blockIdx.x * m + c) * kk + i] = (double)sum;
    }
}

// X[:,c] *= f[c] (device factors).
__global__ void k_scale_cols_dev(int n, int m, double* __restrict__ X, long long ldx, const double* __restrict__ f) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * m) return;
    const int c = (int)(idx / n);
    const long long r = idx % n;
    X[(size_t)c * ldx + r] *= f[c];
}

// Y[:,c] (FP32) = f[c] X[:,c] (FP64): the scaled start vectors of an FP32 inner solve.
__global__ void k_scale_cols_to32(int n, int m, const double* __restrict__ X, long long ldx,
                                  const double* __restrict__ f, float* __restrict__ Y, long long ldy) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * m) return;
    const int c = (int)(idx / n);
    const long long r = idx % n;
    Y[(size_t)c * ldy + r] = (float)(f[c] * X[(size_t)c * ldx + r]);
}

// W[:,c] += sum_{j < ju[c]} T_j[:,c] y[c][j] with the FP32 vectors of an inner
// solve (interleaved, vector j of column c at T + (j m + c) n), FP64 sums.
__global__ void k_gm_accumulate32(int n, int m, const float* __restrict__ T, const double* __restrict__ y, int ldy,
                                  GmSteps ju, double* __restrict__ W, long long ldw) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    for (int c = 0; c < m; ++c) {
        double acc = W[(size_t)c * ldw + r];
        const int jc = ju.v[c];
        for (int j = 0; j < jc; ++j) acc += (double)T[((size_t)j * m + c) * n + r] * y[(size_t)c * ldy + j];
        W[(size_t)c * ldw + r] = acc;
    }
}

// ---------------------------------------------------------------------------
// x-line preconditioner of convection-diffusion.  With the y (and z)
// directions in sine modes, eps K + beta_x Gx (x) M_rest + s M is block
// diagonal: mode (j, k) of the transformed directions carries the 1D matrix
// mu_j mu_k T(m), T(m) = eps Kx + beta_x Gx + m Mx, m = s + eps (lam_j + lam_k)
// (the y, z convection is left out).  T(m) is tridiagonal Toeplitz with
// sub-diagonal a = -eps/h - beta/2 + m h/6, diagonal d = 2 eps/h + 4 m h/6 and
// super-diagonal c = -eps/h + beta/2 + m h/6.  Its symmetric part is positive
// definite, so the pivots of elimination without pivoting stay positive.
// ---------------------------------------------------------------------------

// Thomas factors per mode: IP[i] = 1 / (d - a CP[i-1]), CP[i] = c IP[i].
__global__ void k_line_factor(int nx, int nmodes, int ny, int dim, double hx, double eps, double bx, double shift,
                              const double* __restrict__ lam1, const double* __restrict__ lam2,
                              double* __restrict__ CP64, double* __restrict__ IP64, float* __restrict__ CP32,
                              float* __restrict__ IP32) {
    const int mode = blockIdx.x * blockDim.x + threadIdx.x;
    if (mode >= nmodes) return;
    double mu = shift;
    if (dim > 1) mu += eps * lam1[mode % ny];
    if (dim > 2) mu += eps * lam2[mode / ny];
    const double a = -eps / hx - 0.5 * bx + mu * hx / 6.0;
    const double d = 2.0 * eps / hx + 4.0 * mu * hx / 6.0;
    const double c = -eps / hx + 0.5 * bx + mu * hx / 6.0;
    double cp = 0.0;
    const size_t o = (size_t)mode * nx;
    for (int i = 0; i < nx; ++i) {
        const double ip = 1.0 / (d - a * cp);
        cp = c * ip;
        CP64[o + i] = cp;
        IP64[o + i] = ip;
        CP32[o + i] = (float)cp;
        IP32[o + i] = (float)ip;
    }
}

// One thread per (mode, column) row of nx entries: the right-hand side scaled
// by coef c2_j c2_k (the normalisation of the transformed directions), then
// the forward and backward Thomas sweeps.  dst may equal src.  Consecutive
// threads walk consecutive rows, so each 32-byte sector serves several steps
// from L1.
template <typename T, int LB>
__global__ void k_line_solve(int nx, int nmodes, int ny, int dim, int ncols, const T* src, long long lds, T* dst,
                             long long ldd, const T* __restrict__ CP,
                             const T* __restrict__ IP, double hx, double eps, double bx, double shift,
                             const double* __restrict__ lam1, const double* __restrict__ lam2,
                             const double* __restrict__ c2y, const double* __restrict__ c2z, double coef) {
    const long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= (long long)nmodes * ncols) return;
    const int col = (int)(row / nmodes), mode = (int)(row % nmodes);
    double w = coef, mu = shift;
    if (dim > 1) {
        w *= c2y[mode % ny];
        mu += eps * lam1[mode % ny];
    }
    if (dim > 2) {
        w *= c2z[mode / ny];
        mu += eps * lam2[mode / ny];
    }
    const T wt = (T)w;
    const T a = (T)(-eps / hx - 0.5 * bx + mu * hx / 6.0);   // sub-diagonal of T(mu)
    const T* x = src + (size_t)col * lds + (size_t)mode * nx;
    T* y = dst + (size_t)col * ldd + (size_t)mode * nx;
    const T* cp = CP + (size_t)mode * nx;
    const T* ip = IP + (size_t)mode * nx;
    // The sweeps are chains of dependent FMAs; the operands of LB steps are loaded
    // first so that memory latency is paid once per LB steps, not once per step.
    T dprev = T(0);
    for (int i0 = 0; i0 < nx; i0 += LB) {
        T xv[LB], iv[LB];
#pragma unroll
        for (int u = 0; u < LB; ++u) {
            const int i = i0 + u;
            xv[u] = i < nx ? x[i] : T(0);
            iv[u] = i < nx ? ip[i] : T(0);
        }
#pragma unroll
        for (int u = 0; u < LB; ++u) {
            const int i = i0 + u;
            if (i < nx) {
                dprev = (wt * xv[u] - a * dprev) * iv[u];
                y[i] = dprev;
            }
        }
    }
    T xn = dprev;
    for (int i1 = nx - 2; i1 >= 0; i1 -= LB) {
        T yv[LB], cv[LB];
#pragma unroll
        for (int u = 0; u < LB; ++u) {
            const int i = i1 - u;
            yv[u] = i >= 0 ? y[i] : T(0);
            cv[u] = i >= 0 ? cp[i] : T(0);
        }
#pragma unroll
        for (int u = 0; u < LB; ++u) {
            const int i = i1 - u;
            if (i >= 0) {
                xn = yv[u] - cv[u] * xn;
                y[i] = xn;
            }
        }
    }
}

// Line solves with a warp per row (partition method) for grids with few rows,
// where one sequential thread per row leaves the GPU idle: lane k owns the
// chunk [k L, (k+1) L) of the row (L = ceil(nx/32) <= 8).  Each lane solves
// its chunk's Toeplitz block three times (the leading-block Thomas factors are
// the first entries of the row's factors): y for its right-hand side, v and w
// for the couplings -a and -c to the unknowns left and right of the chunk, so
// x = y + v x_left + w x_right.  The chunks' first and last unknowns then
// satisfy a two-term recurrence over the chunks, run by lane 0 in shared
// memory, and every lane finishes its chunk.
template <typename T>
__global__ void __launch_bounds__(128) k_line_solve_warp(int nx, int nmodes, int ny, int dim, int ncols, const T* src,
                                                         long long lds, T* dst, long long ldd,
                                                         const T* __restrict__ CP, const T* __restrict__ IP,
                                                         double hx, double eps, double bx, double shift,
                                                         const double* __restrict__ lam1,
                                                         const double* __restrict__ lam2,
                                                         const double* __restrict__ c2y,
                                                         const double* __restrict__ c2z, double coef) {
    constexpr int LMAX = 8;
    __shared__ T sh[4][32][6];   // per warp: y, v, w at the chunk ends
    __shared__ T sx[4][33][2];   // per warp: the chunk's first and last unknowns
    const int wib = threadIdx.x / 32, lane = threadIdx.x % 32;
    const long long row = (long long)blockIdx.x * 4 + wib;
    if (row >= (long long)nmodes * ncols) return;   // uniform over the warp
    const int col = (int)(row / nmodes), mode = (int)(row % nmodes);
    double w = coef, mu = shift;
    if (dim > 1) {
        w *= c2y[mode % ny];
        mu += eps * lam1[mode % ny];
    }
    if (dim > 2) {
        w *= c2z[mode / ny];
        mu += eps * lam2[mode / ny];
    }
    const T wt = (T)w;
    const T a = (T)(-eps / hx - 0.5 * bx + mu * hx / 6.0);
    const T cc = (T)(-eps / hx + 0.5 * bx + mu * hx / 6.0);
    const int L = (nx + 31) / 32;
    const int P = (nx + L - 1) / L;   // non-empty chunks
    const int s0 = lane * L;
    const int Lk = lane < P ? min(L, nx - s0) : 0;
    const T* x = src + (size_t)col * lds + (size_t)mode * nx;
    T* out = dst + (size_t)col * ldd + (size_t)mode * nx;
    const T* cp = CP + (size_t)mode * nx;
    const T* ip = IP + (size_t)mode * nx;
    T b[LMAX], y[LMAX], v[LMAX], u[LMAX], cpl[LMAX], ipl[LMAX];
#pragma unroll
    for (int i = 0; i < LMAX; ++i) {
        const bool in = i < Lk;
        b[i] = in ? wt * x[s0 + i] : T(0);
        cpl[i] = in ? cp[i] : T(0);
        ipl[i] = in ? ip[i] : T(0);
    }
    // forward sweeps of the three right-hand sides (b, -a e_1, -c e_Lk)
    T dy = T(0), dv = T(0), du = T(0);
#pragma unroll
    for (int i = 0; i < LMAX; ++i) {
        if (i < Lk) {
            dy = (b[i] - a * dy) * ipl[i];
            dv = ((i == 0 ? -a : T(0)) - a * dv) * ipl[i];
            du = ((i == Lk - 1 ? -cc : T(0)) - a * du) * ipl[i];
            y[i] = dy;
            v[i] = dv;
            u[i] = du;
        }
    }
#pragma unroll
    for (int i = LMAX - 2; i >= 0; --i) {
        if (i < Lk - 1) {
            y[i] -= cpl[i] * y[i + 1];
            v[i] -= cpl[i] * v[i + 1];
            u[i] -= cpl[i] * u[i + 1];
        }
    }
    if (lane < P) {
        sh[wib][lane][0] = y[0];
        sh[wib][lane][1] = y[Lk - 1 < 0 ? 0 : Lk - 1];
        sh[wib][lane][2] = v[0];
        sh[wib][lane][3] = v[Lk - 1 < 0 ? 0 : Lk - 1];
        sh[wib][lane][4] = u[0];
        sh[wib][lane][5] = u[Lk - 1 < 0 ? 0 : Lk - 1];
    }
    __syncwarp();
    if (lane == 0) {
        // g_{k-1} = al + be f_k; f_k = A_k + B_k f_{k+1}; g_k = al_k + be_k f_{k+1}
        T al = T(0), be = T(0);
        T A[32], B[32], AL[32], BE[32];
        for (int k = 0; k < P; ++k) {
            const T yf = sh[wib][k][0], yl = sh[wib][k][1], vf = sh[wib][k][2], vl = sh[wib][k][3];
            const T wf = sh[wib][k][4], wl = sh[wib][k][5];
            const T den = T(1) - vf * be;
            A[k] = (yf + vf * al) / den;
            B[k] = wf / den;
            AL[k] = yl + vl * al + vl * be * A[k];
            BE[k] = vl * be * B[k] + wl;
            al = AL[k];
            be = BE[k];
        }
        T fnext = T(0);   // the unknown right of the last chunk is the boundary
        for (int k = P - 1; k >= 0; --k) {
            const T f = A[k] + B[k] * fnext;
            const T g = AL[k] + BE[k] * fnext;
            sx[wib][k][0] = f;
            sx[wib][k][1] = g;
            fnext = f;
        }
    }
    __syncwarp();
    if (lane < P) {
        const T xl = lane > 0 ? sx[wib][lane - 1][1] : T(0);
        const T xr = lane + 1 < P ? sx[wib][lane + 1][0] : T(0);
#pragma unroll
        for (int i = 0; i < LMAX; ++i)
            if (i < Lk) out[s0 + i] = y[i] + v[i] * xl + u[i] * xr;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// host wrappers
// ---------------------------------------------------------------------------
namespace {
thread_local StTuneSession* t_tune = nullptr;
}

StTuneSession* st_tune_set_session(StTuneSession* sess) {
    StTuneSession* prev = t_tune;
    t_tune = sess;
    return prev;
}

StTuneSession* st_tune_session(cudaStream_t s) {
    if (!t_tune) return nullptr;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();   // the query's error must not surface at a later launch check
        return nullptr;
    }
    return cs == cudaStreamCaptureStatusNone ? t_tune : nullptr;
}

int st_tune_measure(cudaStream_t s, int n, const bool* valid, const std::function<void(int)>& run,
                    const std::function<int()>& prep, double* ms) {
    constexpr int kRounds = 4, kReps = 3;
    std::vector<cudaEvent_t> ev((size_t)2 * kRounds * n * kReps, nullptr);
    int rc = ST_OK;
    for (auto& e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            e = nullptr;
            rc = ST_ECUDA;
        }
    for (int r = 0; r < kRounds && rc == ST_OK; ++r)
        for (int c = 0; c < n && rc == ST_OK; ++c) {
            if (!valid[c]) continue;
            for (int q = 0; q < kReps && rc == ST_OK; ++q) {
                if (prep) rc = prep();
                if (rc != ST_OK) break;
                const size_t i = 2 * (((size_t)r * n + c) * kReps + q);
                cudaEventRecord(ev[i], s);
                run(c);
                st_count_launch();
                if (cudaGetLastError() != cudaSuccess) rc = ST_ECUDA;
                cudaEventRecord(ev[i + 1], s);
            }
        }
    if (rc == ST_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = ST_ECUDA;
    std::vector<double> t((size_t)kRounds * n, -1.0);
    for (int r = 0; r < kRounds && rc == ST_OK; ++r)
        for (int c = 0; c < n; ++c) {
            if (!valid[c]) continue;
            double sum = 0.0;
            for (int q = 0; q < kReps; ++q) {
                const size_t i = 2 * (((size_t)r * n + c) * kReps + q);
                float e = 0.f;
                if (cudaEventElapsedTime(&e, ev[i], ev[i + 1]) != cudaSuccess) {
                    rc = ST_ECUDA;
                    break;
                }
                sum += e;
            }
            t[(size_t)r * n + c] = sum;
        }
    for (auto e : ev)
        if (e) cudaEventDestroy(e);
    if (rc != ST_OK) {
        st_note_msg("autotune: a timed launch failed");
        return rc;
    }
    sttune::reduce_rounds(t.data(), kRounds, n, ms);
    return ST_OK;
}

// 1D factors of the box problem's M and A (see k_apply_sf3): mass h/6 (1, 4, 1),
// stiffness (-1, 2, -1)/h, convection beta_d/2 (-1, 0, 1), as the assembly uses them.
static SfStencil sf_stencil(const st_problem* p) {
    SfStencil f{};
    for (int d = 0; d < 3; ++d) {
        const double h = p->len[d] / (p->n[d] + 1);
        const double k0 = 2.0 / h, k1 = -1.0 / h;
        double am, a0, ap;
        if (p->d.op == ST_CONVDIFF) {
            const double e = p->d.eps, b = p->d.beta[d];
            am = e * k1 - 0.5 * b;
            a0 = e * k0;
            ap = e * k1 + 0.5 * b;
        } else {
            am = ap = p->kappa * k1;
            a0 = p->kappa * k0;
        }
        f.m0[d] = (float)(4.0 * h / 6.0);
        f.m1[d] = (float)(h / 6.0);
        f.am[d] = (float)am;
        f.a0[d] = (float)a0;
        f.ap[d] = (float)ap;
    }
    f.hdt = (float)(0.5 * p->dt);
    return f;
}

template <typename T>
int st_apply_kernel(st_problem* p, const T* U, int ldu, T* Y, int ldy, int n_t, cudaStream_t s) {
    const T* pv;
    const T* nv;
    if constexpr (sizeof(T) == 8) {
        pv = (const T*)p->p64;
        nv = (const T*)p->q64;
    } else {
        pv = (const T*)p->p32;
        nv = (const T*)p->q32;
    }
    if (p->box_ok && (p->dim == 2 || p->dim == 3)) {
        const int nx = p->n[0], ny = p->n[1], nz = p->n[2];
        BoxStencil<T> S;
        for (int e = 0; e < 27; ++e) {
            S.p[e] = (T)(sizeof(T) == 8 ? p->box_p64[e] : p->box_p32[e]);
            S.q[e] = (T)(sizeof(T) == 8 ? p->box_q64[e] : p->box_q32[e]);
        }
        // blocks of 32 x-points by 8 thread rows; each thread YB (x ZB) points and `steps`
        // columns.  FP32: the time-pair kernel in 2D and the sum-factorised kernel in 3D (their
        // own blockings below).  FP64 (FP64-ALU-bound): 2D 4 rows x 8, 3D 2 x 2 x 16.
        const int YB = p->dim == 2 ? 4 : 2, ZB = p->dim == 2 ? 1 : 2;   // FP64 blockings
        long long blocks = (long long)((nx + 31) / 32) * ((ny + 8 * YB - 1) / (8 * YB)) *
                           (p->dim == 3 ? (nz + ZB - 1) / ZB : 1);
        const int steps = p->dim == 2 ? 8 : 16;
        dim3 grid((unsigned)blocks, (unsigned)((n_t + steps - 1) / steps));
        if (sizeof(T) == 8 && (blocks > 0x7fffffffLL || grid.y > 65535)) return ST_EINVAL;
        double ts = (double)sizeof(T);
        st_prof_begin(s, sizeof(T) == 8 ? "apply64" : "apply32", ts * 2.0 * (double)p->n_h * n_t,
                      4.0 * (double)p->max_row_nnz * p->n_h * n_t);
        if constexpr (sizeof(T) == 4) {
            if (p->dim == 2) {
                // 30 x-points by 8 x 4 rows a CTA; 15 time columns (8 pairs, the first starting one
                // column early for N u_{l0-1})
                constexpr int YB2 = 4, NP2 = 8, ST2 = 2 * NP2 - 1;
                const long long b2 = (long long)((nx + 29) / 30) * ((ny + 8 * YB2 - 1) / (8 * YB2));
                const dim3 g2((unsigned)b2, (unsigned)((n_t + ST2 - 1) / ST2));
                if (b2 > 0x7fffffffLL || g2.y > 65535) return ST_EINVAL;
                k_apply_box_tp<YB2, NP2><<<g2, dim3(32, 8), 0, s>>>(nx, ny, n_t, S, (const float*)U, ldu,
                                                                   (float*)Y, ldy);
            } else {
                // sum-factorised: 30 x-points, 8 x 4 rows in y, 6 planes in z a CTA; 16 time columns
                // (the fastest of the blockings measured on 63^3 x 128 and 127^3 x 512)
                constexpr int YB3 = 4, ZB3 = 6, ST3 = 16;
                const long long b3 = (long long)((nx + 29) / 30) * ((ny + 8 * YB3 - 1) / (8 * YB3)) *
                                     ((nz + ZB3 - 1) / ZB3);
                const dim3 g3((unsigned)b3, (unsigned)((n_t + ST3 - 1) / ST3));
                if (b3 > 0x7fffffffLL || g3.y > 65535) return ST_EINVAL;
                k_apply_sf3<YB3, ZB3><<<g3, dim3(32, 8), 0, s>>>(nx, ny, nz, n_t, ST3, sf_stencil(p),
                                                                 (const float*)U, ldu, (float*)Y, ldy);
            }
        } else {
            if (p->dim == 2)
                k_apply_box<T, 2, 4, 1, 8><<<grid, dim3(32, 8), 0, s>>>(nx, ny, nz, n_t, S, U, ldu, Y, ldy);
            else
                k_apply_box<T, 3, 2, 2, 16><<<grid, dim3(32, 8), 0, s>>>(nx, ny, nz, n_t, S, U, ldu, Y, ldy);
        }
        st_prof_end(s);
        ST_LAUNCH_CHECK();
        return ST_OK;
    }
    int rows_blocks = (p->n_h + 127) / 128;
    // split time into chunks so that the grid holds about 300k threads
    long long want = 300000;
    int nchunk = (int)std::min<long long>(n_t, std::max<long long>(1, want / std::max(1, p->n_h)));
    int chunk = (n_t + nchunk - 1) / nchunk;
    nchunk = (n_t + chunk - 1) / chunk;
    dim3 grid(rows_blocks, nchunk);
    double ts = (double)sizeof(T);
    st_prof_begin(s, sizeof(T) == 8 ? "apply64" : "apply32",
                  ts * 2.0 * (double)p->n_h * n_t + (double)p->nnz * (4.0 + 2.0 * ts) + 4.0 * (p->n_h + 1),
                  4.0 * (double)p->nnz * n_t);
    // register buckets of the row length: 3 (1D), 9 (2D P1/Q1), 16 (3D P1 on Kuhn-type meshes: 15), 27 (3D Q1);
    // a padded entry still costs a gather and two FMAs, and the 27-wide FP32 thread held 248 registers
    if (p->max_row_nnz <= 3)
        k_apply_reg<T, 3><<<grid, 128, 0, s>>>(p->n_h, n_t, chunk, p->row_ptr, p->col, pv, nv, U, ldu, Y, ldy);
    else if (p->max_row_nnz <= 9)
        k_apply_reg<T, 9, sizeof(T) == 4 ? 4 : 1><<<grid, 128, 0, s>>>(p->n_h, n_t, chunk, p->row_ptr, p->col, pv, nv,
                                                                        U, ldu, Y, ldy);
    else if (p->max_row_nnz <= 16)
        k_apply_reg<T, 16, sizeof(T) == 4 ? 4 : 1><<<grid, 128, 0, s>>>(p->n_h, n_t, chunk, p->row_ptr, p->col, pv,
                                                                         nv, U, ldu, Y, ldy);
    else if (p->max_row_nnz <= 27)
        k_apply_reg<T, 27><<<grid, 128, 0, s>>>(p->n_h, n_t, chunk, p->row_ptr, p->col, pv, nv, U, ldu, Y, ldy);
    else
        k_apply_generic<T><<<grid, 128, 0, s>>>(p->n_h, n_t, chunk, p->row_ptr, p->col, pv, nv, U, ldu, Y, ldy);
    st_prof_end(s);
    ST_LAUNCH_CHECK();
    return ST_OK;
}
template int st_apply_kernel<double>(st_problem*, const double*, int, double*, int, int, cudaStream_t);
template int st_apply_kernel<float>(st_problem*, const float*, int, float*, int, int, cudaStream_t);

// Launch k_stencil_box over the problem's box grid (2D: 2 points per thread
// in y; 3D: 2 x 2 in y, z).
template <typename T>
static void launch_stencil_box(st_problem* p, const BoxPair<T>& S, const T* X, int ldx, int ncols, T beta, T* O1,
                               int ld1, T* O2, int ld2, cudaStream_t s) {
    const int nx = p->n[0], ny = p->n[1], nz = p->dim == 3 ? p->n[2] : 1;
    const int YB = 2, ZB = p->dim == 2 ? 1 : 2;
    const long long blocks = (long long)((nx + 31) / 32) * ((ny + 8 * YB - 1) / (8 * YB)) * ((nz + ZB - 1) / ZB);
    dim3 grid((unsigned)blocks, (unsigned)ncols);
    if (p->dim == 2)
        k_stencil_box<T, 2, 2, 1><<<grid, dim3(32, 8), 0, s>>>(nx, ny, nz, S, X, ldx, beta, O1, ld1, O2, ld2);
    else
        k_stencil_box<T, 3, 2, 2><<<grid, dim3(32, 8), 0, s>>>(nx, ny, nz, S, X, ldx, beta, O1, ld1, O2, ld2);
}

static bool use_box(const st_problem* p, int ncols) {
    return p->box_ok && (p->dim == 2 || p->dim == 3) && ncols <= 65535;
}

template <typename T>
int st_spmm_ma(st_problem* p, const T* X, int ldx, int ncols, T* OM, int ldm, T* OA, int lda, cudaStream_t s) {
    if (ncols <= 0) return ST_OK;
    const T *mv, *av;
    if constexpr (sizeof(T) == 8) {
        mv = (const T*)p->m64;
        av = (const T*)p->a64;
    } else {
        mv = (const T*)p->m32;
        av = (const T*)p->a32;
    }
    int blocks = (p->n_h + 127) / 128;
    double ts = (double)sizeof(T);
    int nout = (OM ? 1 : 0) + (OA ? 1 : 0);
    if (nout > 0 && use_box(p, ncols)) {
        BoxPair<T> S;
        for (int e = 0; e < 27; ++e) {
            T m = sizeof(T) == 8 ? (T)p->box_m64[e] : (T)p->box_m32[e];
            T a = sizeof(T) == 8 ? (T)p->box_a64[e] : (T)p->box_a32[e];
            S.s[0][e] = OM ? m : a;
            S.s[1][e] = a;
        }
        st_prof_begin(s, sizeof(T) == 8 ? "spmm64_box" : "spmm32_box", ts * (double)p->n_h * ncols * (1 + nout),
                      2.0 * (p->dim == 2 ? 9 : 27) * (double)p->n_h * ncols * nout);
        launch_stencil_box<T>(p, S, X, ldx, ncols, T(0), OM ? OM : OA, OM ? ldm : lda, OM ? OA : nullptr, lda, s);
        st_prof_end(s);
        ST_LAUNCH_CHECK();
        return ST_OK;
    }
    st_prof_begin(s, sizeof(T) == 8 ? "spmm64" : "spmm32",
                  (double)p->nnz * (4.0 + 2.0 * ts) + 4.0 * (p->n_h + 1) + ts * (double)p->n_h * ncols * (1 + nout),
                  4.0 * (double)p->nnz * ncols);
    if (p->max_row_nnz <= 3)
        k_spmm_ma_reg<T, 3><<<blocks, 128, 0, s>>>(p->n_h, ncols, p->row_ptr, p->col, mv, av, X, ldx, OM, ldm, OA, lda);
    else if (p->max_row_nnz <= 9)
        k_spmm_ma_reg<T, 9><<<blocks, 128, 0, s>>>(p->n_h, ncols, p->row_ptr, p->col, mv, av, X, ldx, OM, ldm, OA, lda);
    else if (p->max_row_nnz <= 16)   // 3D P1 rows (15 entries on Kuhn-type meshes)
        k_spmm_ma_reg<T, 16><<<blocks, 128, 0, s>>>(p->n_h, ncols, p->row_ptr, p->col, mv, av, X, ldx, OM, ldm, OA, lda);
    else if (p->max_row_nnz <= 27)
        k_spmm_ma_reg<T, 27><<<blocks, 128, 0, s>>>(p->n_h, ncols, p->row_ptr, p->col, mv, av, X, ldx, OM, ldm, OA, lda);
    else
        k_spmm_ma_generic<T><<<blocks, 128, 0, s>>>(p->n_h, ncols, p->row_ptr, p->col, mv, av, X, ldx, OM, ldm, OA, lda);
    st_prof_end(s);
    ST_LAUNCH_CHECK();
    return ST_OK;
}
template int st_spmm_ma<double>(st_problem*, const double*, int, int, double*, int, double*, int, cudaStream_t);
template int st_spmm_ma<float>(st_problem*, const float*, int, int, float*, int, float*, int, cudaStream_t);

int st_spmm_at64(st_problem* p, const double* X, int ldx, int ncols, double* Out, int ldo, cudaStream_t s) {
    if (ncols <= 0) return ST_OK;
    if (!p->at64) return ST_ENOTSUP;
    if (use_box(p, ncols)) {
        // a constant stencil's transpose is the stencil reflected through its centre
        BoxPair<double> S;
        for (int e = 0; e < 27; ++e) S.s[0][e] = S.s[1][e] = p->box_a64[26 - e];
        st_prof_begin(s, "spmm_at64_box", 16.0 * (double)p->n_h * ncols,
                      2.0 * (p->dim == 2 ? 9 : 27) * (double)p->n_h * ncols);
        launch_stencil_box<double>(p, S, X, ldx, ncols, 0.0, Out, ldo, nullptr, 0, s);
        st_prof_end(s);
        ST_LAUNCH_CHECK();
        return ST_OK;
    }
    int blocks = (p->n_h + 127) / 128;
    st_prof_begin(s, "spmm_at64", (double)p->nnz * 12.0 + 4.0 * (p->n_h + 1) + 16.0 * (double)p->n_h * ncols,
                  2.0 * (double)p->nnz * ncols);
    if (p->max_row_nnz <= 3)
        k_spmm_ma_reg<double, 3><<<blocks, 128, 0, s>>>(p->n_h, ncols, p->row_ptr, p->col, p->at64, p->at64, X, ldx,
                                                         Out, ldo, nullptr, 0);
    else if (p->max_row_nnz <= 9)
        k_spmm_ma_reg<double, 9><<<blocks, 128, 0, s>>>(p->n_h, ncols, p->row_ptr, p->col, p->at64, p->at64, X, ldx,
                                                         Out, ldo, nullptr, 0);
    else if (p->max_row_nnz <= 16)
        k_spmm_ma_reg<double, 16><<<blocks, 128, 0, s>>>(p->n_h, ncols, p->row_ptr, p->col, p->at64, p->at64, X, ldx,
                                                          Out, ldo, nullptr, 0);
    else if (p->max_row_nnz <= 27)
        k_spmm_ma_reg<double, 27><<<blocks, 128, 0, s>>>(p->n_h, ncols, p->row_ptr, p->col, p->at64, p->at64, X, ldx,
                                                          Out, ldo, nullptr, 0);
    else
        k_spmm_ma_generic<double><<<blocks, 128, 0, s>>>(p->n_h, ncols, p->row_ptr, p->col, p->at64, p->at64, X, ldx,
                                                          Out, ldo, nullptr, 0);
    st_prof_end(s);
    ST_LAUNCH_CHECK();
    return ST_OK;
}

int st_spmm_comb64(st_problem* p, double cm, double ca, const double* X, int ldx, int ncols, double beta, double* Out,
                   int ldo, cudaStream_t s) {
    if (ncols <= 0) return ST_OK;
    if (use_box(p, ncols)) {
        BoxPair<double> S;
        for (int e = 0; e < 27; ++e) S.s[0][e] = S.s[1][e] = cm * p->box_m64[e] + ca * p->box_a64[e];
        st_prof_begin(s, "spmm_comb64_box", 8.0 * (double)p->n_h * ncols * (beta == 0.0 ? 2 : 3),
                      2.0 * (p->dim == 2 ? 9 : 27) * (double)p->n_h * ncols);
        launch_stencil_box<double>(p, S, X, ldx, ncols, beta, Out, ldo, nullptr, 0, s);
        st_prof_end(s);
        ST_LAUNCH_CHECK();
        return ST_OK;
    }
    int blocks = (p->n_h + 127) / 128;
    st_prof_begin(s, "spmm_comb64", (double)p->nnz * 20.0 + 4.0 * (p->n_h + 1) + 8.0 * p->n_h * ncols * (beta == 0.0 ? 2 : 3),
                  4.0 * (double)p->nnz * ncols);
    k_spmm_comb64<<<blocks, 128, 0, s>>>(p->n_h, ncols, p->row_ptr, p->col, p->m64, p->a64, cm, ca, X, ldx, beta, Out, ldo);
    st_prof_end(s);
    ST_LAUNCH_CHECK();
    return ST_OK;
}

int st_cn_rhs_step(st_problem* p, const double* u, const double* F1, int ldf1, const double* F2, int ldf2, int l,
                   int ncols, double* out, cudaStream_t s) {
    int blocks = (p->n_h + 127) / 128;
    if (u && use_box(p, 1)) {
        // box grid: the load term first, then N u from the constant stencil added onto it
        st_prof_begin(s, "cn_rhs_box", 8.0 * p->n_h * (3 + ncols), 2.0 * (p->dim == 2 ? 9 : 27) * p->n_h);
        k_cn_rhs<<<blocks, 128, 0, s>>>(p->n_h, p->row_ptr, p->col, p->q64, nullptr, F1, ldf1, F2, ldf2, l, ncols,
                                        out);
        ST_LAUNCH_CHECK();
        BoxPair<double> S;
        for (int e = 0; e < 27; ++e) S.s[0][e] = S.s[1][e] = p->box_q64[e];
        launch_stencil_box<double>(p, S, u, p->n_h, 1, 1.0, out, p->n_h, nullptr, 0, s);
        st_prof_end(s);
        ST_LAUNCH_CHECK();
        return ST_OK;
    }
    st_prof_begin(s, "cn_rhs", (double)p->nnz * 12.0 + 4.0 * (p->n_h + 1) + 8.0 * p->n_h * (2 + ncols),
                  2.0 * (double)p->nnz + 2.0 * p->n_h * ncols);
    k_cn_rhs<<<blocks, 128, 0, s>>>(p->n_h, p->row_ptr, p->col, p->q64, u, F1, ldf1, F2, ldf2, l, ncols, out);
    st_prof_end(s);
    ST_LAUNCH_CHECK();
    return ST_OK;
}

// Fast diagonalisation W = coef * Q(x) diag(omega) Q(x) X on the tensor grid.
// The vector of one column is the tensor X[z][y][x] (x fastest).  Forward
// products run over x, y, z; the spectral weights are applied in the epilogue
// of the last forward product; the backward products reuse Q (symmetric).
// Every product handles all columns in one launch.  Buffers alternate
// X -> tmp -> W -> tmp -> ... so that the last product lands in W (2*dim
// products); X is read only by the first, so X and W may alias.
template <typename T>
static int fd_apply_impl(st_problem* p, FdKind kind, double shift, double coef, const T* X, int ldx, int ncols, T* W,
                         int ldw, T* tmp, cudaStream_t s, const T* const* Q, const T* const (*HG)[4],
                         const char* tag) {
    int dim = p->dim;
    int nx = p->n[0], ny = p->n[1], nz = p->n[2];
    long long nh = p->n_h;
    FdEpi plain{};
    plain.scale = 0;
    plain.coef = 1.0;
    FdEpi sc{};
    sc.scale = 1;
    sc.dim = dim;
    sc.nx = nx;
    sc.ny = ny;
    sc.nz = nz;
    sc.l0 = p->ax[0].lam;
    sc.l1 = dim > 1 ? p->ax[1].lam : p->ax[0].lam;
    sc.l2 = dim > 2 ? p->ax[2].lam : p->ax[0].lam;
    sc.c0 = p->ax[0].c2;
    sc.c1 = dim > 1 ? p->ax[1].c2 : p->ax[0].c2;
    sc.c2 = dim > 2 ? p->ax[2].c2 : p->ax[0].c2;
    sc.f0 = p->ax[0].lam32;
    sc.f1 = dim > 1 ? p->ax[1].lam32 : p->ax[0].lam32;
    sc.f2 = dim > 2 ? p->ax[2].lam32 : p->ax[0].lam32;
    sc.g0 = p->ax[0].c232;
    sc.g1 = dim > 1 ? p->ax[1].c232 : p->ax[0].c232;
    sc.g2 = dim > 2 ? p->ax[2].c232 : p->ax[0].c232;
    sc.kind = kind;
    sc.kappa = p->fd_kappa;
    sc.shift = shift;
    sc.coef = 1.0;
    if (kind == FD_MASS_RESOLVENT)
        for (int d = 0; d < dim; ++d) sc.coef *= 2.0 / (p->n[d] + 1);
    FdEpi fin = plain;
    fin.coef = coef;
    const T* src = X;
    long long lds = ldx;
    T* bufs[2] = {tmp, W};
    long long ldb[2] = {nh, ldw};
    int step = 0;
    for (int pass = 0; pass < 2; ++pass) {
        for (int d = 0; d < dim; ++d) {
            T* dst = bufs[step % 2];
            long long ldd = ldb[step % 2];
            bool last_fwd = (pass == 0 && d == dim - 1);
            bool last_all = (pass == 1 && d == dim - 1);
            FdEpi ep = last_fwd ? sc : (last_all ? fin : plain);
            if (d == 0) {
                long long R = nh / nx;
                ep.left = 0;
                ep.J = 1;
                Batch2 bt{1, 0, lds, 0, 0, 0, ldd};   // one batch per column: z2 = column
                (void)Q;
                ST_TRY((launch_gemm_fold<T, 0>(nx, (int)R, src, nx, HG[0], dst, nx, ncols, bt, ep, s, tag)));
            } else {
                long long J = (d == 1) ? nx : (long long)nx * ny;
                int nd = p->n[d];
                int outer = (int)(nh / (J * nd));
                ep.left = 1;
                ep.J = J;
                Batch2 bt{outer, 0, 0, (long long)nd * J, lds, (long long)nd * J, ldd};
                ST_TRY((launch_gemm_fold<T, 1>(nd, (int)J, src, J, HG[d], dst, J, outer * ncols, bt, ep, s, tag)));
            }
            src = dst;
            lds = ldd;
            ++step;
        }
    }
    return ST_OK;
}

int st_fd_apply64(st_problem* p, FdKind kind, double shift, double coef, const double* X, int ldx, int ncols,
                  double* W, int ldw, double* tmp, cudaStream_t s) {
    if (p->dim < 1) return ST_ENOTSUP;
    const double* Q[3] = {p->ax[0].Q64, p->ax[1].Q64, p->ax[2].Q64};
    const double* HG[3][4];
    for (int d = 0; d < 3; ++d)
        for (int t = 0; t < 4; ++t) HG[d][t] = p->ax[d].fold64[t];
    return fd_apply_impl<double>(p, kind, shift, coef, X, ldx, ncols, W, ldw, tmp, s, Q, HG, "fd_gemm64");
}

int st_fd_apply32(st_problem* p, FdKind kind, double shift, double coef, const float* X, int ldx, int ncols, float* W,
                  int ldw, float* tmp, cudaStream_t s) {
    if (p->dim < 1) return ST_ENOTSUP;
    const float* Q[3] = {p->ax[0].Q32, p->ax[1].Q32, p->ax[2].Q32};
    const float* HG[3][4];
    for (int d = 0; d < 3; ++d)
        for (int t = 0; t < 4; ++t) HG[d][t] = p->ax[d].fold32[t];
    return fd_apply_impl<float>(p, kind, shift, coef, X, ldx, ncols, W, ldw, tmp, s, Q, HG, "fd_gemm32");
}

bool st_line_usable(const st_problem* p) {
    if (p->d.op != ST_CONVDIFF || p->dim < 1 || p->dim > 3 || !(p->d.eps > 0)) return false;
    const double bx = std::fabs(p->d.beta[0]);
    for (int d = 1; d < p->dim; ++d)
        if (std::fabs(p->d.beta[d]) > bx) return false;
    return true;
}

int st_line_factor(st_problem* p, double shift, cudaStream_t s) {
    if (!st_line_usable(p)) return ST_ENOTSUP;
    if (p->line_valid && p->line_shift == shift) return ST_OK;
    const size_t nh = (size_t)p->n_h;
    if (!p->line_cp64) {
        ST_TRY(st_alloc(p, (void**)&p->line_cp64, sizeof(double) * nh));
        ST_TRY(st_alloc(p, (void**)&p->line_ip64, sizeof(double) * nh));
        ST_TRY(st_alloc(p, (void**)&p->line_cp32, sizeof(float) * nh));
        ST_TRY(st_alloc(p, (void**)&p->line_ip32, sizeof(float) * nh));
    }
    const int nx = p->n[0];
    const int ny = p->dim > 1 ? p->n[1] : 1;
    const int nmodes = (int)(nh / nx);
    k_line_factor<<<(nmodes + 127) / 128, 128, 0, s>>>(nx, nmodes, ny, p->dim, p->ax[0].h, p->d.eps, p->d.beta[0],
                                                      shift, p->dim > 1 ? p->ax[1].lam : nullptr,
                                                      p->dim > 2 ? p->ax[2].lam : nullptr, p->line_cp64,
                                                      p->line_ip64, p->line_cp32, p->line_ip32);
    ST_LAUNCH_CHECK();
    p->line_shift = shift;
    p->line_valid = true;
    return ST_OK;
}

// y (and z) forward transforms, the x line solves, the backward transforms:
// 2D X -> tmp -> (solve in place) -> W; 3D X -> tmp -> W -> (solve) -> tmp -> W;
// 1D the solve alone, X -> W.
template <typename T>
static int line_apply_impl(st_problem* p, double coef, const T* X, int ldx, int ncols, T* W, int ldw, T* tmp,
                           cudaStream_t s, const T* const (*HG)[4], const T* CP, const T* IP, const char* tag) {
    if (!p->line_valid) return ST_EINVAL;
    const int dim = p->dim, nx = p->n[0], ny = dim > 1 ? p->n[1] : 1;
    const long long nh = p->n_h;
    const int nmodes = (int)(nh / nx);
    const double hx = p->ax[0].h, eps = p->d.eps, bx = p->d.beta[0];
    FdEpi plain{};
    plain.scale = 0;
    plain.coef = 1.0;
    auto transform = [&](int d, const T* src, long long lds, T* dst, long long ldd) -> int {
        const long long J = (d == 1) ? nx : (long long)nx * ny;
        const int nd = p->n[d];
        const int outer = (int)(nh / (J * nd));
        FdEpi ep = plain;
        ep.left = 1;
        ep.J = J;
        Batch2 bt{outer, 0, 0, (long long)nd * J, lds, (long long)nd * J, ldd};
        return launch_gemm_fold<T, 1>(nd, (int)J, src, J, HG[d], dst, J, outer * ncols, bt, ep, s, tag);
    };
    auto solve = [&](const T* src, long long lds, T* dst, long long ldd) -> int {
        const long long rows = (long long)nmodes * ncols;
        const double* l1 = dim > 1 ? p->ax[1].lam : nullptr;
        const double* l2 = dim > 2 ? p->ax[2].lam : nullptr;
        const double* g1 = dim > 1 ? p->ax[1].c2 : nullptr;
        const double* g2 = dim > 2 ? p->ax[2].c2 : nullptr;
        // variants: 0 a warp per row (partition method, rows of at most 256 points);
        // 1 a thread per row, loads in batches of 64 steps; 2 the same with 16 steps
        // (fewer registers on many rows)
        auto go = [&](int c) {
            if (c == 0)
                k_line_solve_warp<T><<<(unsigned)((rows + 3) / 4), 128, 0, s>>>(
                    nx, nmodes, ny, dim, ncols, src, lds, dst, ldd, CP, IP, hx, eps, bx, p->line_shift, l1, l2, g1,
                    g2, coef);
            else if (c == 1)
                k_line_solve<T, 64><<<(unsigned)((rows + 63) / 64), 64, 0, s>>>(
                    nx, nmodes, ny, dim, ncols, src, lds, dst, ldd, CP, IP, hx, eps, bx, p->line_shift, l1, l2, g1,
                    g2, coef);
            else
                k_line_solve<T, 16><<<(unsigned)((rows + 127) / 128), 128, 0, s>>>(
                    nx, nmodes, ny, dim, ncols, src, lds, dst, ldd, CP, IP, hx, eps, bx, p->line_shift, l1, l2, g1,
                    g2, coef);
        };
        // built-in choice: few rows (a 2D grid: N_y p) and short rows take a warp per row
        // (2D 255^2: 58 -> 13 us a launch; on 63^3, 7938 rows, the thread per row is
        // faster); the sweeps are latency-bound, so each batch of loads covers 64 steps,
        // except FP64 on many rows: 16, which keeps the registers below 128
        const int def = (rows < 2048 && nx <= 256) ? 0 : ((rows < 8192 || sizeof(T) == 4) ? 1 : 2);
        const sttune::Key key{sttune::LINE, (int)sizeof(T), nx, (int)std::min<long long>(rows, 1LL << 30), dim, 0};
        int c = sttune::table().get(key);
        const size_t col_bytes = sizeof(T) * (size_t)nh;
        const bool in_place = (const void*)src == (const void*)dst;
        StTuneSession* ts = c < 0 ? st_tune_session(s) : nullptr;
        if (ts && (!in_place || ts->scratch_bytes >= col_bytes * ncols)) {
            // an in-place solve is timed on a saved copy of its input, restored before
            // every launch and once more before the launch that counts
            std::function<int()> restore;
            if (in_place) {
                ST_CUDA_TRY(cudaMemcpy2DAsync(ts->scratch, col_bytes, src, sizeof(T) * lds, col_bytes, ncols,
                                              cudaMemcpyDeviceToDevice, s));
                restore = [&]() -> int {
                    ST_CUDA_TRY(cudaMemcpy2DAsync(dst, sizeof(T) * ldd, ts->scratch, col_bytes, col_bytes, ncols,
                                                  cudaMemcpyDeviceToDevice, s));
                    return ST_OK;
                };
            }
            bool valid[3] = {nx <= 256, true, true};
            double ms[3];
            ST_TRY(st_tune_measure(s, 3, valid, go, restore, ms));
            c = sttune::pick(ms, 3, def, 0.03);
            sttune::table().put(key, c);
            ++ts->tuned;
            if (in_place) ST_TRY(restore());
        }
        if (c < 0 || (c == 0 && nx > 256)) c = def;
        st_prof_begin(s, sizeof(T) == 8 ? "line64" : "line32", 4.0 * sizeof(T) * (double)nh * ncols,
                      5.0 * (double)nh * ncols);
        go(c);
        st_prof_end(s);
        ST_LAUNCH_CHECK();
        return ST_OK;
    };
    if (dim == 1) return solve(X, ldx, W, ldw);
    if (dim == 2) {
        ST_TRY(transform(1, X, ldx, tmp, nh));
        ST_TRY(solve(tmp, nh, tmp, nh));
        return transform(1, tmp, nh, W, ldw);
    }
    ST_TRY(transform(1, X, ldx, tmp, nh));
    ST_TRY(transform(2, tmp, nh, W, ldw));
    ST_TRY(solve(W, ldw, W, ldw));
    ST_TRY(transform(1, W, ldw, tmp, nh));
    return transform(2, tmp, nh, W, ldw);
}

int st_line_apply64(st_problem* p, double coef, const double* X, int ldx, int ncols, double* W, int ldw, double* tmp,
                    cudaStream_t s) {
    const double* HG[3][4];
    for (int d = 0; d < 3; ++d)
        for (int t = 0; t < 4; ++t) HG[d][t] = p->ax[d].fold64[t];
    return line_apply_impl<double>(p, coef, X, ldx, ncols, W, ldw, tmp, s, HG, p->line_cp64, p->line_ip64,
                                   "fd_gemm64");
}

int st_line_apply32(st_problem* p, double coef, const float* X, int ldx, int ncols, float* W, int ldw, float* tmp,
                    cudaStream_t s) {
    const float* HG[3][4];
    for (int d = 0; d < 3; ++d)
        for (int t = 0; t < 4; ++t) HG[d][t] = p->ax[d].fold32[t];
    return line_apply_impl<float>(p, coef, X, ldx, ncols, W, ldw, tmp, s, HG, p->line_cp32, p->line_ip32,
                                  "fd_gemm32");
}

size_t st_tsgemm_partial_elems(int n, int k, int m) {
    // the largest partial buffer any column chunk of at most kMaxCols needs
    int mm = m < kMaxCols ? m : kMaxCols;
    size_t nch = (size_t)((n + ts_rows(n, k, mm) - 1) / ts_rows(n, k, mm));
    size_t nch1 = (size_t)((n + ts_rows(n, k, 1) - 1) / ts_rows(n, k, 1));
    return (nch > nch1 ? nch : nch1) * (size_t)k * (size_t)mm;
}

namespace {
// Launch the templated kernel whose MAXM (2, 4, 8 or 16) covers m.
template <template <int> class L, typename... Args>
void dispatch_m(int m, Args... args) {
    if (m <= 2) L<2>::go(args...);
    else if (m <= 4) L<4>::go(args...);
    else if (m <= 8) L<8>::go(args...);
    else L<16>::go(args...);
}

template <int MAXM> struct LaunchTn {
    static void go(dim3 grid, size_t smem, cudaStream_t s, int n, int k, int m, int rows, const double* V, int ldv,
                   const double* W, int ldw, double* part) {
        static const bool set = [] {
            cudaFuncSetAttribute(k_ts_tn_partial<MAXM>, cudaFuncAttributeMaxDynamicSharedMemorySize, 8192 * 8);
            return true;
        }();
        (void)set;
        k_ts_tn_partial<MAXM><<<grid, TS_THREADS, smem, s>>>(n, k, m, rows, V, ldv, W, ldw, part);
    }
};
template <int MAXM> struct LaunchTnDf {
    static void go(dim3 grid, size_t smem, cudaStream_t s, int n, int k, int m, int rows, const float2* V, int ldv,
                   const float2* W, int ldw, float2* part, bool hi) {
        static const bool set = [] {
            cudaFuncSetAttribute(k_ts_tn_df_partial<MAXM, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 8192 * 8);
            cudaFuncSetAttribute(k_ts_tn_df_partial<MAXM, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 8192 * 8);
            return true;
        }();
        (void)set;
        if (hi)
            k_ts_tn_df_partial<MAXM, true><<<grid, TS_THREADS, smem, s>>>(n, k, m, rows, V, ldv, W, ldw, part);
        else
            k_ts_tn_df_partial<MAXM, false><<<grid, TS_THREADS, smem, s>>>(n, k, m, rows, V, ldv, W, ldw, part);
    }
};
template <int MAXM> struct LaunchNn {
    static void go(int blocks, cudaStream_t s, int n, int k, int m, double alpha, const double* V, int ldv,
                   const double* H, int ldh, double beta, double* W, int ldw) {
        k_ts_nn<MAXM><<<blocks, 256, 0, s>>>(n, k, m, alpha, V, ldv, H, ldh, beta, W, ldw);
    }
};
template <int MAXM> struct LaunchNnDf {
    static void go(int blocks, cudaStream_t s, int n, int k, int m, double alpha, const float2* V, int ldv,
                   const double* H, int ldh, double beta, double* W, int ldw) {
        k_ts_nn_df<MAXM><<<blocks, 256, 0, s>>>(n, k, m, alpha, V, ldv, H, ldh, beta, W, ldw);
    }
};
}  // namespace

int st_tsgemm_tn(int n, int k, int m, const double* V, int ldv, const double* W, int ldw, double* H, int ldh,
                 double* partial, cudaStream_t s) {
    if (k <= 0 || m <= 0) return ST_OK;
    if (m > kMaxCols) {   // wider blocks in chunks of kMaxCols columns
        for (int j0 = 0; j0 < m; j0 += kMaxCols) {
            int mm = m - j0 < kMaxCols ? m - j0 : kMaxCols;
            ST_TRY(st_tsgemm_tn(n, k, mm, V, ldv, W + (size_t)j0 * ldw, ldw, H + (size_t)j0 * ldh, ldh, partial, s));
        }
        return ST_OK;
    }
    if (n <= 0) {
        // empty sum
        for (int b = 0; b < m; ++b) ST_CUDA_TRY(cudaMemsetAsync(H + (size_t)b * ldh, 0, sizeof(double) * k, s));
        return ST_OK;
    }
    const int rows = ts_rows(n, k, m);
    const int nch = (n + rows - 1) / rows;
    const size_t smem = sizeof(double) * (size_t)m * rows;
    dim3 grid(nch, (k + TS_CG - 1) / TS_CG);
    if (grid.y > 65535) return ST_EINVAL;
    st_prof_begin(s, "ts_tn", 8.0 * (double)n * (k + m) + 16.0 * (double)nch * k * m, 2.0 * (double)n * k * m);
    dispatch_m<LaunchTn>(m, grid, smem, s, n, k, m, rows, V, ldv, W, ldw, partial);
    ST_LAUNCH_CHECK();
    k_ts_reduce<<<(k * m + 7) / 8, 256, 0, s>>>(nch, k, m, partial, H, ldh);
    st_prof_end(s);
    ST_LAUNCH_CHECK();
    return ST_OK;
}

int st_tsgemm_nn(int n, int k, int m, double alpha, const double* V, int ldv, const double* H, int ldh, double beta,
                 double* W, int ldw, cudaStream_t s) {
    if (n <= 0 || m <= 0) return ST_OK;
    if (m > kMaxCols) {   // wider blocks in chunks of kMaxCols columns
        for (int j0 = 0; j0 < m; j0 += kMaxCols) {
            int mm = m - j0 < kMaxCols ? m - j0 : kMaxCols;
            ST_TRY(st_tsgemm_nn(n, k, mm, alpha, V, ldv, H + (size_t)j0 * ldh, ldh, beta, W + (size_t)j0 * ldw, ldw, s));
        }
        return ST_OK;
    }
    if (k <= 0) {
        if (beta == 1.0) return ST_OK;
        return st_axpby64(n, m, 0.0, W, ldw, beta, W, ldw, s);
    }
    st_prof_begin(s, "ts_nn", 8.0 * (double)n * (k + m * (beta == 0.0 ? 1 : 2)), 2.0 * (double)n * k * m);
    dispatch_m<LaunchNn>(m, (n + 255) / 256, s, n, k, m, alpha, V, ldv, H, ldh, beta, W, ldw);
    st_prof_end(s);
    ST_LAUNCH_CHECK();
    return ST_OK;
}

int st_to_df(int n, int m, const double* X, int ldx, float2* Y, int ldy, cudaStream_t s) {
    long long tot = (long long)n * m;
    if (tot <= 0) return ST_OK;
    k_to_df<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(n, m, X, ldx, Y, ldy);
    ST_LAUNCH_CHECK();
    return ST_OK;
}

int st_tsgemm_tn_df(int n, int k, int m, const float2* V, int ldv, const float2* W, int ldw, double* H, int ldh,
                    double* partial, cudaStream_t s, bool hi_only) {
    if (k <= 0 || m <= 0) return ST_OK;
    if (m > kMaxCols) {   // wider blocks in chunks of kMaxCols columns
        for (int j0 = 0; j0 < m; j0 += kMaxCols) {
            int mm = m - j0 < kMaxCols ? m - j0 : kMaxCols;
            ST_TRY(st_tsgemm_tn_df(n, k, mm, V, ldv, W + (size_t)j0 * ldw, ldw, H + (size_t)j0 * ldh, ldh, partial, s,
                                   hi_only));
        }
        return ST_OK;
    }
    if (n <= 0) {
        for (int b = 0; b < m; ++b) ST_CUDA_TRY(cudaMemsetAsync(H + (size_t)b * ldh, 0, sizeof(double) * k, s));
        return ST_OK;
    }
    const int rows = ts_rows(n, k, m);
    const int nch = (n + rows - 1) / rows;
    const size_t smem = sizeof(float4) * (size_t)((m + 1) / 2) * rows;   // column pairs, at most 64 KB
    dim3 grid(nch, (k + TS_CG_DF - 1) / TS_CG_DF);
    if (grid.y > 65535) return ST_EINVAL;
    float2* part2 = reinterpret_cast<float2*>(partial);   // (hi, lo) pairs in the doubles' room
    st_prof_begin(s, hi_only ? "ts_tn_hi" : "ts_tn_df", 8.0 * (double)n * (k + m) + 16.0 * (double)nch * k * m,
                  2.0 * (double)n * k * m);
    dispatch_m<LaunchTnDf>(m, grid, smem, s, n, k, m, rows, V, ldv, W, ldw, part2, hi_only);
    ST_LAUNCH_CHECK();
    k_ts_reduce_df<<<(k * m + 7) / 8, 256, 0, s>>>(nch, k, m, part2, H, ldh);
    st_prof_end(s);
    ST_LAUNCH_CHECK();
    return ST_OK;
}

int st_tsgemm_nn_df(int n, int k, int m, double alpha, const float2* V, int ldv, const double* H, int ldh,
                    double beta, double* W, int ldw, cudaStream_t s) {
    if (n <= 0 || m <= 0) return ST_OK;
    if (m > kMaxCols) {   // wider blocks in chunks of kMaxCols columns
        for (int j0 = 0; j0 < m; j0 += kMaxCols) {
            int mm = m - j0 < kMaxCols ? m - j0 : kMaxCols;
            ST_TRY(st_tsgemm_nn_df(n, k, mm, alpha, V, ldv, H + (size_t)j0 * ldh, ldh, beta, W + (size_t)j0 * ldw, ldw, s));
        }
        return ST_OK;
    }
    if (k <= 0) {
        if (beta == 1.0) return ST_OK;
        return st_axpby64(n, m, 0.0, W, ldw, beta, W, ldw, s);
    }
    st_prof_begin(s, "ts_nn_df", 8.0 * (double)n * (k + m * (beta == 0.0 ? 1 : 2)), 2.0 * (double)n * k * m);
    dispatch_m<LaunchNnDf>(m, (n + 255) / 256, s, n, k, m, alpha, V, ldv, H, ldh, beta, W, ldw);
    st_prof_end(s);
    ST_LAUNCH_CHECK();
    return ST_OK;
}

int st_trsm_right_upper(int n, int m, const double* R, int ldr, double* W, int ldw, cudaStream_t s) {
    if (n <= 0 || m <= 0) return ST_OK;
    if (m > kMaxCols) return ST_EINVAL;
    k_trsm_right_upper<<<(n + 255) / 256, 256, 0, s>>>(n, m, R, ldr, W, ldw);
    ST_LAUNCH_CHECK();
    return ST_OK;
}

int st_chol_small(int m, const double* G, int ldg, double* R, int ldr, double* flag, cudaStream_t s) {
    if (m <= 0) return ST_OK;
    if (m > kMaxCols) return ST_EINVAL;
    k_chol_small<<<1, 32, 0, s>>>(m, G, ldg, R, ldr, flag);
    ST_LAUNCH_CHECK();
    return ST_OK;
}

int st_copy_cols64(int n, int m, const double* X, int ldx, double* Y, int ldy, cudaStream_t s) {
    long long tot = (long long)n * m;
    if (tot <= 0) return ST_OK;
    k_copy_cols<double, double><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(n, m, X, ldx, Y, ldy, 0.0);
    ST_LAUNCH_CHECK();
    return ST_OK;
}

int st_convert_64_32(int n, int m, const double* X, int ldx, float* Y, int ldy, cudaStream_t s) {
    long long tot = (long long)n * m;
    if (tot <= 0) return ST_OK;
    k_copy_cols<double, float><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(n, m, X, ldx, Y, ldy, 0.0);
    ST_LAUNCH_CHECK();
    return ST_OK;
}

int st_convert_32_64_add(int n, int m, const float* X, int ldx, double* Y, int ldy, double beta, cudaStream_t s) {
    long long tot = (long long)n * m;
    if (tot <= 0) return ST_OK;
    k_copy_cols<float, double><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(n, m, X, ldx, Y, ldy, beta);
    ST_LAUNCH_CHECK();
    return ST_OK;
}

int st_axpby64(int n, int m, double a, const double* X, int ldx, double b, double* Y, int ldy, cudaStream_t s) {
    long long tot = (long long)n * m;
    if (tot <= 0) return ST_OK;
    k_axpby<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(n, m, a, X, ldx, b, Y, ldy);
    ST_LAUNCH_CHECK();
    return ST_OK;
}

// C (r x c, column-major) = X (r x s) Y (s x c): as the row-major product C^T = Y^T X^T.
int st_gemm_cm(int r, int c, int s, const double* X, int ldx, const double* Y, int ldy, double* C, int ldc,
               cudaStream_t st) {
    FdEpi plain{};
    plain.coef = 1.0;
    Batch2 bt{1, 0, 0, 0, 0, 0, 0};
    return launch_gemm_rr<double>(c, r, s, Y, ldy, X, ldx, C, ldc, 1, bt, plain, st, "dense_gemm");
}

// U (n x n_t, col-major) = V (n x k) Y (k x n_t): as row-major U^T = Y^T V^T.
int st_lowrank_dense(int n, int k, int n_t, const double* V, int ldv, const double* Y, int ldy, double* U, int ldu,
                     cudaStream_t s) {
    FdEpi plain{};
    plain.coef = 1.0;
    if (k == 0) {
        for (int l = 0; l < n_t; ++l) ST_CUDA_TRY(cudaMemsetAsync(U + (size_t)l * ldu, 0, sizeof(double) * n, s));
        return ST_OK;
    }
    Batch2 bt{1, 0, 0, 0, 0, 0, 0};
    return launch_gemm_rr<double>(n_t, n, k, Y, ldy, V, ldv, U, ldu, 1, bt, plain, s, "lowrank_gemm");
}

// ---------------------------------------------------------------------------
// batched flexible GMRES building blocks
// ---------------------------------------------------------------------------
static int gm_rows(int n, int m) {
    // about 600 CTAs over the m columns, 256..4096 rows a chunk
    long long nch = std::max(1, 608 / std::max(1, m));
    long long rows = (n + nch - 1) / nch;
    rows = (rows + 31) / 32 * 32;
    return (int)std::min<long long>(4096, std::max<long long>(256, rows));
}

// Chunk rows of the fused update-and-dots kernel: as gm_rows, but the chunk's
// new vectors (m x rows of T) must fit in 160 KB of shared memory.
static int gm_rows_ud(int n, int m, size_t tsize) {
    const int cap = (int)((160 * 1024) / ((size_t)m * tsize)) / 32 * 32;
    return std::max(32, std::min(gm_rows(n, m), cap));
}

size_t st_gm_partial_elems(int n, int kk, int m) {
    // the larger chunk count of the two partitions (the fused one at its FP64 worst case)
    const int r1 = gm_rows(n, m), r2 = gm_rows_ud(n, m, sizeof(double));
    const size_t nch = (size_t)std::max((n + r1 - 1) / r1, (n + r2 - 1) / r2);
    return nch * (size_t)m * (size_t)kk;
}

template <typename T>
int st_gm_dots(int n, int kk, int m, const T* Z, double* part, double* H, int ldh, cudaStream_t s) {
    if (n <= 0 || kk <= 0 || m <= 0 || m > kMaxCols) return ST_EINVAL;
    const int rows = gm_rows(n, m);
    const int nch = (n + rows - 1) / rows;
    st_prof_begin(s, sizeof(T) == 8 ? "gm_dot" : "gm_dot32",
                  (double)sizeof(T) * n * kk * m + 16.0 * (double)nch * kk * m, 2.0 * (double)n * kk * m);
    k_gm_dot_partial<T><<<dim3(nch, m), 256, sizeof(T) * rows, s>>>(n, kk, m, rows, Z, part);
    ST_LAUNCH_CHECK();
    k_gm_reduce<<<(kk * m + 7) / 8, 256, 0, s>>>(nch, kk, m, part, H, ldh);
    st_prof_end(s);
    ST_LAUNCH_CHECK();
    return ST_OK;
}

template int st_gm_dots<double>(int, int, int, const double*, double*, double*, int, cudaStream_t);
template int st_gm_dots<float>(int, int, int, const float*, double*, double*, int, cudaStream_t);

template <typename T>
int st_gm_update(int n, int nb, int m, T* Z, const double* H, int ldh, const double* H1, int ldh1, double* Hd,
                 long long ldhd, int jcol, int J, cudaStream_t s) {
    if (n <= 0 || nb < 0 || m <= 0 || m > kMaxCols) return ST_EINVAL;
    const int blocks = (n + 255) / 256;
    const size_t smem = sizeof(double) * ((size_t)m * (nb + 1) + m) + sizeof(T) * (size_t)m * (nb + 1);
    st_prof_begin(s, sizeof(T) == 8 ? "gm_update" : "gm_update32", (double)sizeof(T) * n * m * (nb + 2),
                  2.0 * (double)n * m * nb);
    if (m <= 1)
        k_gm_update<T, 1><<<blocks, 256, smem, s>>>(n, nb, m, Z, H, ldh, H1, ldh1, Hd, ldhd, jcol, J);
    else if (m <= 2)
        k_gm_update<T, 2><<<blocks, 256, smem, s>>>(n, nb, m, Z, H, ldh, H1, ldh1, Hd, ldhd, jcol, J);
    else if (m <= 4)
        k_gm_update<T, 4><<<blocks, 256, smem, s>>>(n, nb, m, Z, H, ldh, H1, ldh1, Hd, ldhd, jcol, J);
    else if (m <= 8)
        k_gm_update<T, 8><<<blocks, 256, smem, s>>>(n, nb, m, Z, H, ldh, H1, ldh1, Hd, ldhd, jcol, J);
    else
        k_gm_update<T, 16><<<blocks, 256, smem, s>>>(n, nb, m, Z, H, ldh, H1, ldh1, Hd, ldhd, jcol, J);
    st_prof_end(s);
    ST_LAUNCH_CHECK();
    return ST_OK;
}

template <typename T, int MAXM>
static void launch_update_dot(int nch, size_t smem, cudaStream_t s, int n, int nb, int m, int rows, T* Z,
                              const double* H, int ldh, double* part) {
    static const bool set = [] {
        cudaFuncSetAttribute(k_gm_update_dot<T, MAXM>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        return true;
    }();
    (void)set;
    k_gm_update_dot<T, MAXM><<<nch, 256, smem, s>>>(n, nb, m, rows, Z, H, ldh, part);
}

template <typename T>
int st_gm_update_dot(int n, int nb, int m, T* Z, const double* H1, int ldh1, double* part, double* H2, int ldh2,
                     cudaStream_t s) {
    if (n <= 0 || nb < 0 || m <= 0 || m > kMaxCols) return ST_EINVAL;
    const int rows = gm_rows_ud(n, m, sizeof(T));
    const int nch = (n + rows - 1) / rows;
    const int kk = nb + 1;
    const size_t smem = sizeof(double) * (size_t)m * kk + sizeof(T) * ((size_t)m * kk + (size_t)m * rows);
    if (smem > 200 * 1024) return ST_EINVAL;
    st_prof_begin(s, sizeof(T) == 8 ? "gm_update_dot" : "gm_update_dot32",
                  (double)sizeof(T) * n * m * (nb + 2) + 16.0 * (double)nch * kk * m, 4.0 * (double)n * m * kk);
    if (m <= 1)
        launch_update_dot<T, 1>(nch, smem, s, n, nb, m, rows, Z, H1, ldh1, part);
    else if (m <= 2)
        launch_update_dot<T, 2>(nch, smem, s, n, nb, m, rows, Z, H1, ldh1, part);
    else if (m <= 4)
        launch_update_dot<T, 4>(nch, smem, s, n, nb, m, rows, Z, H1, ldh1, part);
    else if (m <= 8)
        launch_update_dot<T, 8>(nch, smem, s, n, nb, m, rows, Z, H1, ldh1, part);
    else
        launch_update_dot<T, 16>(nch, smem, s, n, nb, m, rows, Z, H1, ldh1, part);
    ST_LAUNCH_CHECK();
    k_gm_reduce<<<(kk * m + 7) / 8, 256, 0, s>>>(nch, kk, m, part, H2, ldh2);
    st_prof_end(s);
    ST_LAUNCH_CHECK();
    return ST_OK;
}
template int st_gm_update_dot<double>(int, int, int, double*, const double*, int, double*, double*, int,
                                      cudaStream_t);
template int st_gm_update_dot<float>(int, int, int, float*, const double*, int, double*, double*, int, cudaStream_t);

template int st_gm_update<double>(int, int, int, double*, const double*, int, const double*, int, double*, long long,
                                  int, int, cudaStream_t);
template int st_gm_update<float>(int, int, int, float*, const double*, int, const double*, int, double*, long long,
                                 int, int, cudaStream_t);

int st_scale_cols_to32(int n, int m, const double* X, int ldx, const double* f, float* Y, int ldy, cudaStream_t s) {
    if (n <= 0 || m <= 0) return ST_OK;
    const long long tot = (long long)n * m;
    k_scale_cols_to32<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(n, m, X, ldx, f, Y, ldy);
    ST_LAUNCH_CHECK();
    return ST_OK;
}

int st_gm_accumulate32(int n, int m, const float* T, const double* y, int ldy, const GmSteps& ju, double* W, int ldw,
                       cudaStream_t s) {
    if (n <= 0 || m <= 0) return ST_OK;
    if (m > 16) return ST_EINVAL;
    st_prof_begin(s, "gm_accumulate32", 4.0 * (double)n * m * 40 + 16.0 * (double)n * m, 2.0 * (double)n * m * 40);
    k_gm_accumulate32<<<(n + 255) / 256, 256, 0, s>>>(n, m, T, y, ldy, ju, W, ldw);
    st_prof_end(s);
    ST_LAUNCH_CHECK();
    return ST_OK;
}

int st_spmm_comb32(st_problem* p, double cm, double ca, const float* X, int ldx, int ncols, float* Out, int ldo,
                   cudaStream_t s) {
    if (ncols <= 0) return ST_OK;
    if (!use_box(p, ncols)) return ST_ENOTSUP;
    BoxPair<float> S;
    for (int e = 0; e < 27; ++e) S.s[0][e] = S.s[1][e] = (float)(cm * p->box_m64[e] + ca * p->box_a64[e]);
    st_prof_begin(s, "spmm_comb32_box", 8.0 * (double)p->n_h * ncols, 2.0 * (p->dim == 2 ? 9 : 27) * (double)p->n_h * ncols);
    // shuffle kernel: 4 y-rows (2D) or 4 x 2 (y, z) points a thread, 30 outputs a warp row
    const int nx = p->n[0], ny = p->n[1], nz = p->dim == 3 ? p->n[2] : 1;
    const int YB = 4, ZB = p->dim == 2 ? 1 : 2;
    const long long blocks = (long long)((nx + 29) / 30) * ((ny + 8 * YB - 1) / (8 * YB)) * ((nz + ZB - 1) / ZB);
    dim3 grid((unsigned)blocks, (unsigned)ncols);
    if (p->dim == 2)
        k_stencil_box_sh<2, 4, 1><<<grid, dim3(32, 8), 0, s>>>(nx, ny, nz, S, X, ldx, 0.f, Out, ldo);
    else
        k_stencil_box_sh<3, 4, 2><<<grid, dim3(32, 8), 0, s>>>(nx, ny, nz, S, X, ldx, 0.f, Out, ldo);
    st_prof_end(s);
    ST_LAUNCH_CHECK();
    return ST_OK;
}

int st_scale_cols_dev(int n, int m, double* X, int ldx, const double* f, cudaStream_t s) {
    if (n <= 0 || m <= 0) return ST_OK;
    const long long tot = (long long)n * m;
    k_scale_cols_dev<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(n, m, X, ldx, f);
    ST_LAUNCH_CHECK();
    return ST_OK;
}
