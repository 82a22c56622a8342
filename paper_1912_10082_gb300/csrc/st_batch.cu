// Batched RKSM (paper Section 4, heat): many independent problems solved in
// lock step, every device step of an iteration issued as ONE grouped launch
// over all instances still iterating (st_group.h), with one host
// synchronisation per phase for the whole batch instead of one per instance.
//
// Each instance follows exactly the single-problem driver (solve_impl in
// st_solve.cu): the same host decisions (rank compression, block QR plans,
// adaptive shifts, residual checks) from the same device products, and the
// grouped launches run the tile bodies of the single-problem kernels.  So an
// instance's result does not depend on the other instances of the batch.
//
// Per iteration (instances that still iterate):
//   phase A  shifted solves (fast diagonalisation, FP64 or FP32 refined in
//            FP64) and block CGS2 (FP64 or double-float)      -> one download
//   host     Gram matrices -> rank and first CholQR factor (rare blocks: the
//            column-wise fallback of block_qr, run per instance)
//   phase B  CholQR2 finished on the device, [M q, A q], the products with
//            the basis and with F1                            -> one download
//   phase C  (instances at a residual check) the Gram matrix of the rank-p
//            residual direction, while the host runs the projected solves
//            of those instances                               -> one download
// Host work of an iteration runs on a pool of host threads, one instance per
// item.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <thread>
#include <vector>

#include "st_common.cuh"
#include "st_dev.cuh"
#include "st_group.h"
#include "st_rksm.h"

using namespace rksm;

namespace {

// ---- batch staging: one download region and one upload region for all instances ----
// The device buffer is stream-ordered and the pinned mirror comes from the library's pool, so growing or
// releasing them never waits for the other solves on the device.
struct BStage {
    double* d = nullptr;   // device: [down cap | up cap]
    double* h = nullptr;   // pinned mirror
    size_t cap = 0, down = 0, up = 0, hbytes = 0;
    cudaStream_t s_ = nullptr;
    ~BStage() {
        if (s_) cudaStreamSynchronize(s_);   // the last copies have landed
        if (d) cudaFreeAsync(d, s_);
        st_pinned_put(h, hbytes);
    }
    // room for need doubles in each region; the stream is idle between phases
    int reserve(size_t need, cudaStream_t s) {
        down = up = 0;
        if (need <= cap) return ST_OK;
        ST_CUDA_TRY(cudaStreamSynchronize(s));
        if (d) cudaFreeAsync(d, s);
        st_pinned_put(h, hbytes);
        d = nullptr;
        h = nullptr;
        cap = hbytes = 0;
        s_ = s;
        const size_t c = std::max<size_t>(need + need / 2, 1 << 14);
        cudaError_t e = cudaMallocAsync((void**)&d, sizeof(double) * 2 * c, s);
        if (e == cudaSuccess) {
            h = (double*)st_pinned_get(sizeof(double) * 2 * c, &hbytes);
            if (!h) e = cudaErrorMemoryAllocation;
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            st_note_cuda(e, "batch staging", __FILE__, __LINE__);
            return ST_ENOMEM;
        }
        cap = c;
        return ST_OK;
    }
    // reserve() sized every phase for its total, so these stay in bounds
    double* out(size_t m) {
        double* p = d + down;
        down += pad32(m);
        return p;
    }
    double* in(const double* src, size_t m) {
        double* hp = h + cap + up;
        std::memcpy(hp, src, sizeof(double) * m);
        double* p = d + cap + up;
        up += pad32(m);
        return p;
    }
    const double* host_of(const double* dp) const { return h + (dp - d); }
    int push(cudaStream_t s) {
        if (up) ST_CUDA_TRY(cudaMemcpyAsync(d + cap, h + cap, sizeof(double) * up, cudaMemcpyHostToDevice, s));
        return ST_OK;
    }
    int fetch(cudaStream_t s) {
        if (down) ST_CUDA_TRY(cudaMemcpyAsync(h, d, sizeof(double) * down, cudaMemcpyDeviceToHost, s));
        ST_CUDA_TRY(cudaStreamSynchronize(s));
        return ST_OK;
    }
};

// ---- one instance ----
struct BI {
    st_problem* p = nullptr;
    cudaStream_t own_stream = nullptr;
    Ctx c{};
    int n = 0, nt = 0, prec = 0;
    double dt = 0.0, tol = 0.0;
    bool df = false;
    const double* F1 = nullptr;
    const double* F2 = nullptr;
    int ldf1 = 0, ldf2 = 0, p0 = 0;
    st_solution* sol = nullptr;
    st_stats S{};
    Clock::time_point t0;
    int status = ST_ENOTCONV;
    bool live = true;   // still iterating
    // rank compression
    double *F1d = nullptr, *F1c = nullptr, *dGF = nullptr, *dF2 = nullptr;
    std::vector<double> F2h, R1, T1, Q2, F2c, Ub, sb, Vbt;
    int r1 = 0, src_cols = 0, r = 0;
    bool gram = false;
    double normF = 0.0;
    // basis and projected problem
    int k = 0, pmax = 0;
    double *MV = nullptr, *MAq = nullptr;
    HostSym Mm, Am, Hb;
    std::vector<double> Gm;
    int ldg = 0;
    std::vector<int> boff, bsz, hist_it;
    std::vector<double> shifts, ritz, Y, hist_res;
    int last_ritz_k = -1, it = 0, next_check = 1, mu_extra = 0;
    double res = 1.0;
    bool have_y = false;   // Y belongs to the current basis
    // current iteration
    double s = 0.0;
    int pl = 0, lo = 0, kk = 0, pn = 0, pn_prev = 0;
    double* W = nullptr;
    double *dh[2] = {}, *dG = nullptr, *dG2 = nullptr, *dR2 = nullptr, *dflag = nullptr, *dX12 = nullptr,
           *dX3 = nullptr, *dGb = nullptr;
    QrPlan qp;
    bool explicit_gram = false;
    std::vector<double> Hcol, Gw, Rq, X1, X2, X3, Vw, negR;
    double ref2 = 0.0;
    bool check = false;
    bool aborted = false;   // ended by an error return of the single driver: no output
    void fail(int st) {
        status = st;
        live = false;
        aborted = true;
    }
};

constexpr int kNmaq = 2;   // [M q, A q] (heat: A symmetric)

// The 2 dim mode products of one fast-diagonalisation transform
// W = coef Q(x) diag(omega) Q(x) X (the launches of st_fd_apply64/32), in order,
// with the side (0: x direction, 1: y, z) of each.
template <typename T>
void fd_steps(const st_problem* p, FdKind kind, double shift, double coef, const T* X, int ldx, int ncols, T* W,
              int ldw, T* tmp, std::vector<stg::FoldTask>& out, std::vector<int>& side) {
    const int dim = p->dim, nx = p->n[0], ny = p->n[1], nz = p->n[2];
    const long long nh = p->n_h;
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
    for (int pass = 0; pass < 2; ++pass)
        for (int d = 0; d < dim; ++d) {
            T* dst = bufs[step % 2];
            const long long ldd = ldb[step % 2];
            const bool last_fwd = pass == 0 && d == dim - 1, last_all = pass == 1 && d == dim - 1;
            FdEpi ep = last_fwd ? sc : (last_all ? fin : plain);
            stg::FoldTask t{};
            const void* const* hg = sizeof(T) == 8 ? (const void* const*)p->ax[d].fold64 : (const void* const*)p->ax[d].fold32;
            for (int q = 0; q < 4; ++q) t.HG[q] = hg[q];
            t.X = src;
            t.C = dst;
            int M, N, batch;
            if (d == 0) {
                ep.left = 0;
                ep.J = 1;
                t.n = nx;
                t.other = (int)(nh / nx);
                t.ldx = nx;
                t.ldc = nx;
                t.bt = Batch2{1, 0, lds, 0, 0, 0, ldd};
                batch = ncols;
                M = t.other;
                N = (nx + 1) / 2;
            } else {
                const long long J = d == 1 ? nx : (long long)nx * ny;
                const int nd = p->n[d];
                const int outer = (int)(nh / (J * nd));
                ep.left = 1;
                ep.J = J;
                t.n = nd;
                t.other = (int)J;
                t.ldx = J;
                t.ldc = J;
                t.bt = Batch2{outer, 0, 0, (long long)nd * J, lds, (long long)nd * J, ldd};
                batch = outer * ncols;
                M = (nd + 1) / 2;
                N = (int)J;
            }
            t.ep = ep;
            // the single-problem launch's tile choice (so a problem's result does not depend on the path)
            t.tc = sizeof(T) == 4 && fold_tc_default(t.n, t.other, batch) ? 1 : 0;
            // FP32 SIMT: the 64 x 64 vector-read tile for every problem (small problems leave part of a tile
            // idle, but one launch serves the whole step: the tile shape does not change a result)
            t.tm = sizeof(T) == 4 ? 4 : 2;
            const int ex = t.tc ? FTC_N : 16 * t.tm, ey = t.tc ? FTC_M : 16 * t.tm;
            t.gx = (N + ex - 1) / ex;
            t.gy = (M + ey - 1) / ey;
            t.gz = 2 * batch;
            out.push_back(t);
            side.push_back(d == 0 ? 0 : 1);
            src = dst;
            lds = ldd;
            ++step;
        }
}

// Collects the fold steps of several instances' transforms and issues them
// step by step (one or two grouped launches per step: x direction and y/z).
struct FdBatch {
    int tsize;
    std::vector<std::vector<stg::FoldTask>> steps;   // per instance
    std::vector<std::vector<int>> sides;
    explicit FdBatch(int ts) : tsize(ts) {}
    template <typename T>
    void add(const st_problem* p, FdKind kind, double shift, double coef, const T* X, int ldx, int ncols, T* W,
             int ldw, T* tmp) {
        steps.emplace_back();
        sides.emplace_back();
        fd_steps<T>(p, kind, shift, coef, X, ldx, ncols, W, ldw, tmp, steps.back(), sides.back());
    }
    void issue(stg::GroupPhase& ph) {
        size_t nst = 0;
        for (auto& s : steps) nst = std::max(nst, s.size());
        for (size_t j = 0; j < nst; ++j) {
            std::vector<stg::FoldTask> t0, t1;
            for (size_t i = 0; i < steps.size(); ++i)
                if (j < steps[i].size()) (sides[i][j] == 0 ? t0 : t1).push_back(steps[i][j]);
            ph.fold(tsize, 0, t0);
            ph.fold(tsize, 1, t1);
        }
        steps.clear();
        sides.clear();
    }
};

// Box-stencil task of st_spmm_ma / st_spmm_comb64 on the problem's grid.
stg::StencilTask stencil_task(const st_problem* p, const BoxPair<double>& S, const double* X, int ldx, int ncols,
                              double beta, double* O1, int ld1, double* O2, int ld2) {
    stg::StencilTask t{};
    t.nx = p->n[0];
    t.ny = p->n[1];
    t.nz = p->dim == 3 ? p->n[2] : 1;
    const int YB = 2, ZB = p->dim == 2 ? 1 : 2;
    t.blocks = ((t.nx + 31) / 32) * ((t.ny + 8 * YB - 1) / (8 * YB)) * ((t.nz + ZB - 1) / ZB);
    t.ncols = ncols;
    t.S = S;
    t.X = X;
    t.ldx = ldx;
    t.beta = beta;
    t.O1 = O1;
    t.ld1 = ld1;
    t.O2 = O2;
    t.ld2 = ld2;
    return t;
}

// [M X, A X] (st_spmm_ma with both outputs)
stg::StencilTask ma_task(const st_problem* p, const double* X, int ldx, int ncols, double* OM, double* OA, int ld) {
    BoxPair<double> S;
    for (int e = 0; e < 27; ++e) {
        S.s[0][e] = p->box_m64[e];
        S.s[1][e] = p->box_a64[e];
    }
    return stencil_task(p, S, X, ldx, ncols, 0.0, OM, ld, OA, ld);
}

// Out = (cm M + ca A) X + beta Out (st_spmm_comb64)
stg::StencilTask comb_task(const st_problem* p, double cm, double ca, const double* X, int ldx, int ncols,
                           double beta, double* Out, int ldo) {
    BoxPair<double> S;
    for (int e = 0; e < 27; ++e) S.s[0][e] = S.s[1][e] = cm * p->box_m64[e] + ca * p->box_a64[e];
    return stencil_task(p, S, X, ldx, ncols, beta, Out, ldo, nullptr, 0);
}

// Partial-sum room of H = V^T W over all column chunks of at most 16 (st_tsgemm_tn's split).
size_t tn_part_elems(int n, int k, int m) {
    size_t tot = 0;
    for (int j0 = 0; j0 < m; j0 += kMaxCols) {
        const int mm = std::min(kMaxCols, m - j0);
        const int rows = ts_rows(n, k, mm);
        tot += (size_t)((n + rows - 1) / rows) * k * mm;
    }
    return tot;
}

// H = V^T W (k x m): one task per chunk of at most 16 columns, each with its own partial room.
void tn_tasks(int n, int k, int m, const void* V, int ldv, const void* W, int ldw, bool df, double* part, double* H,
              int ldh, std::vector<stg::TnTask>& out) {
    size_t off = 0;
    for (int j0 = 0; j0 < m; j0 += kMaxCols) {
        const int mm = std::min(kMaxCols, m - j0);
        stg::TnTask t{};
        t.n = n;
        t.k = k;
        t.m = mm;
        t.rows = ts_rows(n, k, mm);
        t.nch = (n + t.rows - 1) / t.rows;
        t.V = V;
        t.ldv = ldv;
        const size_t esz = df ? sizeof(float2) : sizeof(double);
        t.W = (const char*)W + esz * (size_t)j0 * ldw;
        t.ldw = ldw;
        t.part = part + off;
        t.H = H + (size_t)j0 * ldh;
        t.ldh = ldh;
        off += (size_t)t.nch * k * mm;
        out.push_back(t);
    }
}

// W = beta W + alpha V H (k > 0), chunks of at most 16 columns.
void nn_tasks(int n, int k, int m, double alpha, const void* V, int ldv, const double* H, int ldh, double beta,
              double* W, int ldw, std::vector<stg::NnTask>& out) {
    for (int j0 = 0; j0 < m; j0 += kMaxCols) {
        stg::NnTask t{};
        t.n = n;
        t.k = k;
        t.m = std::min(kMaxCols, m - j0);
        t.alpha = alpha;
        t.V = V;
        t.ldv = ldv;
        t.H = H + (size_t)j0 * ldh;
        t.ldh = ldh;
        t.beta = beta;
        t.W = W + (size_t)j0 * ldw;
        t.ldw = ldw;
        out.push_back(t);
    }
}

stg::ElemTask elem(int op, int n, int m, const void* X, int ldx, void* Y, int ldy, double a = 0.0, double b = 0.0) {
    stg::ElemTask t{};
    t.op = op;
    t.n = n;
    t.m = m;
    t.X = X;
    t.ldx = ldx;
    t.Y = Y;
    t.ldy = ldy;
    t.a = a;
    t.b = b;
    return t;
}

// Grows a handle slot; returns its pointer.
template <typename T>
int slot(st_problem* p, int id, size_t elems, T** out) {
    return st_slot(p, id, sizeof(T) * std::max<size_t>(elems, 1), (void**)out);
}


// Device steps of one or more shifted solves W = (A + s M)^{-1} M X of
// several instances (shifted_solve in st_solve.cu), grouped launch by launch:
// FP64 instances run one transform; mixed ones an FP32 transform refined once
// by the FP64 residual r = M X - (A + s M) W.  The same structure serves the
// start block's M^{-1} X (mass_inverse: two refinement steps).
struct SolveLaunches {
    FdBatch fd64{8}, fd32a{4}, fd32b{4};
    std::vector<stg::ElemTask> to32a, add32a, axpby, to32b, add32b;
    std::vector<stg::StencilTask> comb[4];   // by dimension
    void issue(stg::GroupPhase& ph) {
        ph.elem(to32a);
        fd64.issue(ph);
        fd32a.issue(ph);
        ph.elem(add32a);
        ph.stencil(2, comb[2]);
        ph.stencil(3, comb[3]);
        ph.elem(axpby);
        ph.elem(to32b);
        fd32b.issue(ph);
        ph.elem(add32b);
        to32a.clear();
        add32a.clear();
        axpby.clear();
        to32b.clear();
        add32b.clear();
        comb[2].clear();
        comb[3].clear();
    }
};

// W = (A + s M)^{-1} M X for `ncols` columns of instance b; MX = M X.
int add_resolvent(BI& b, double s, const double* X, const double* MX, int ncols, double* W, SolveLaunches& L) {
    st_problem* p = b.p;
    const int n = b.n;
    const size_t nm = (size_t)n * ncols;
    if (b.prec == ST_FP64) {
        double* tmp;
        ST_TRY(slot(p, S_TMP, nm, &tmp));
        L.fd64.add<double>(p, FD_MASS_RESOLVENT, s, 1.0, X, n, ncols, W, n, tmp);
        return ST_OK;
    }
    float *x32, *w32, *t32;
    double* r64;
    ST_TRY(slot(p, S_X32, nm, &x32));
    ST_TRY(slot(p, S_W32, nm, &w32));
    ST_TRY(slot(p, S_T32, nm, &t32));
    ST_TRY(slot(p, S_TMP, nm, &r64));
    L.to32a.push_back(elem(stg::E_TO32, n, ncols, X, n, x32, n));
    L.fd32a.add<float>(p, FD_MASS_RESOLVENT, s, 1.0, x32, n, ncols, w32, n, t32);
    L.add32a.push_back(elem(stg::E_ADD32, n, ncols, w32, n, W, n, 0.0, 0.0));
    L.comb[p->dim].push_back(comb_task(p, -s, -1.0, W, n, ncols, 0.0, r64, n));
    L.axpby.push_back(elem(stg::E_AXPBY, n, ncols, MX, n, r64, n, 1.0, 1.0));
    L.to32b.push_back(elem(stg::E_TO32, n, ncols, r64, n, x32, n));
    L.fd32b.add<float>(p, FD_RESOLVENT, s, 1.0, x32, n, ncols, w32, n, t32);
    L.add32b.push_back(elem(stg::E_ADD32, n, ncols, w32, n, W, n, 0.0, 1.0));
    return ST_OK;
}

// Host half of the rank compression before a possible block QR of F1 (solve_impl, A1).
void compress_plan(BI& b, const double* gf) {
    const int p0 = b.p0, nt = b.nt;
    b.F2h.assign((size_t)nt * p0, 0.0);
    if (b.dF2) {
        std::memcpy(b.F2h.data(), gf + (b.dF2 - b.dGF), sizeof(double) * (size_t)nt * p0);
    } else {
        for (int j = 0; j < p0; ++j) std::memcpy(&b.F2h[(size_t)j * nt], b.F2 + (size_t)j * b.ldf2, sizeof(double) * nt);
    }
    bool finite = true;
    for (size_t i = 0; i < (size_t)p0 * p0; ++i) finite = finite && std::isfinite(gf[i]);
    for (double v : b.F2h) finite = finite && std::isfinite(v);
    if (!finite) {
        st_note_msg("st_solve_batch: F1 or F2 holds a NaN or Inf (or F1^T F1 overflows)");
        b.fail(ST_EINVAL);
        return;
    }
    b.R1.assign((size_t)p0 * p0, 0.0);
    std::vector<double> E(gf, gf + (size_t)p0 * p0), w(p0);
    dense::sym_eig(p0, E.data(), p0, w.data());
    const double wmax = std::max(w[p0 - 1], 0.0);
    b.r1 = 0;
    for (int i = 0; i < p0; ++i) b.r1 += (wmax > 0.0 && w[i] > 1e-28 * wmax);
    b.gram = b.r1 > 0 && w[p0 - b.r1] > 1e-8 * wmax;
    if (b.gram) {
        b.T1.assign((size_t)p0 * b.r1, 0.0);
        for (int t = 0; t < b.r1; ++t) {
            const int e = p0 - b.r1 + t;
            const double sw = std::sqrt(w[e]);
            for (int q = 0; q < p0; ++q) {
                b.R1[(size_t)q * p0 + t] = sw * E[(size_t)e * p0 + q];
                b.T1[(size_t)t * p0 + q] = E[(size_t)e * p0 + q] / sw;
            }
        }
        b.src_cols = p0;
    }
}

// Host half after it: QR of F2, SVD of the small core, kept rank r, F2c and the
// combination Tc with F1c = (F1 or Q1) Tc.
void compress_finish(BI& b, std::vector<double>& Tc) {
    const int p0 = b.p0, nt = b.nt, r1 = b.r1;
    b.Q2 = b.F2h;
    std::vector<double> R2((size_t)p0 * p0);
    dense::thin_qr(nt, p0, b.Q2.data(), nt, R2.data(), p0);
    std::vector<double> B((size_t)r1 * p0, 0.0);
    for (int j = 0; j < p0; ++j)
        for (int i = 0; i < r1; ++i) {
            double s = 0.0;
            for (int q = 0; q < p0; ++q) s += b.R1[(size_t)q * p0 + i] * R2[(size_t)q * p0 + j];
            B[(size_t)j * r1 + i] = s;
        }
    b.r = 0;
    if (r1 > 0) {
        std::vector<double> Bt((size_t)p0 * r1);
        for (int j = 0; j < p0; ++j)
            for (int i = 0; i < r1; ++i) Bt[(size_t)i * p0 + j] = B[(size_t)j * r1 + i];
        std::vector<double> U2((size_t)p0 * r1), s2(r1), V2t((size_t)r1 * r1);
        dense::svd_small(p0, r1, Bt.data(), p0, U2.data(), s2.data(), V2t.data());
        for (int i = 0; i < r1; ++i)
            if (s2[i] > 1e-14 * s2[0]) ++b.r;
        const int r = b.r;
        b.Ub.assign((size_t)r1 * r, 0.0);
        for (int j = 0; j < r; ++j)
            for (int i = 0; i < r1; ++i) b.Ub[(size_t)j * r1 + i] = V2t[(size_t)i * r1 + j];
        b.sb.assign(s2.begin(), s2.begin() + r);
        b.Vbt.assign((size_t)p0 * r, 0.0);
        for (int j = 0; j < r; ++j)
            for (int i = 0; i < p0; ++i) b.Vbt[(size_t)j * p0 + i] = U2[(size_t)j * p0 + i];
    }
    b.normF = 0.0;
    for (double v : b.sb) b.normF += v * v;
    b.normF = std::sqrt(b.normF);
    b.S.p = b.r;
    const int r = b.r;
    if (r == 0) return;
    Tc.assign((size_t)b.src_cols * r, 0.0);
    for (int j = 0; j < r; ++j)
        for (int t = 0; t < r1; ++t) {
            const double u = b.Ub[(size_t)j * r1 + t];
            for (int q = 0; q < b.src_cols; ++q) Tc[(size_t)j * b.src_cols + q] += b.T1[(size_t)t * b.src_cols + q] * u;
        }
    b.F2c.assign((size_t)nt * r, 0.0);
    for (int j = 0; j < r; ++j)
        for (int i = 0; i < nt; ++i) {
            double s = 0.0;
            for (int q = 0; q < p0; ++q) s += b.Q2[(size_t)q * nt + i] * b.Vbt[(size_t)j * p0 + q];
            b.F2c[(size_t)j * nt + i] = s * b.sb[j];
        }
}

// Rank-p residual of a check (solve_impl, A7): ||R||^2 = sum_l g_l^T Gb g_l.
double residual_norm2(BI& b, const double* Gb, bool* ok) {
    const int k = b.k, pl = b.pl, nt = b.nt;
    std::vector<double> H((size_t)k * k), f((size_t)k * pl, 0.0);
    for (int j = 0; j < k; ++j)
        for (int i = 0; i < k; ++i) H[(size_t)j * k + i] = b.Hb(i, j);
    std::vector<int> piv(k);
    dense::lu(k, H.data(), k, piv.data());
    for (int j = 0; j < pl; ++j) f[(size_t)j * k + b.lo + j] = 1.0;
    *ok = dense::lu_solve_transpose(k, H.data(), k, piv.data(), f.data(), k, pl);
    if (!*ok) return 0.0;
    double rr = 0.0;
    std::vector<double> gl(pl);
    for (int l = 0; l < nt; ++l) {
        const double* y = &b.Y[(size_t)l * k];
        const double* yp = l > 0 ? &b.Y[(size_t)(l - 1) * k] : nullptr;
        for (int j = 0; j < pl; ++j) {
            double sacc = 0.0;
            const double* fj = &f[(size_t)j * k];
            for (int i = 0; i < k; ++i) sacc += fj[i] * (y[i] + (yp ? yp[i] : 0.0));
            gl[j] = 0.5 * b.dt * sacc;
        }
        for (int a = 0; a < pl; ++a)
            for (int c = 0; c < pl; ++c) rr += gl[a] * Gb[(size_t)c * pl + a] * gl[c];
    }
    return rr;
}

// Host inputs of the residual direction's Gram product (residual_gram_explicit):
// negR = -R_q (pn x pl) and Vw = Mm^{-1} (s X1_M + X1_A)(-R_q) (k x pl).
bool residual_inputs(BI& b) {
    const int k = b.k, pn = b.pn, pl = b.pl;
    b.negR.assign((size_t)pn * pl, 0.0);
    for (int j = 0; j < pl; ++j)
        for (int i = 0; i < pn; ++i) b.negR[(size_t)j * pn + i] = -b.Rq[(size_t)j * pl + i];
    b.Vw.assign((size_t)k * pl, 0.0);
    for (int j = 0; j < pl; ++j)
        for (int q = 0; q < pn; ++q) {
            const double rq = -b.Rq[(size_t)j * pl + q];
            for (int i = 0; i < k; ++i)
                b.Vw[(size_t)j * k + i] += (b.s * b.X1[(size_t)q * k + i] + b.X1[(size_t)(pn + q) * k + i]) * rq;
        }
    std::vector<double> L((size_t)k * k);
    for (int j = 0; j < k; ++j)
        for (int i = 0; i < k; ++i) L[(size_t)j * k + i] = b.Mm.a[(size_t)j * b.Mm.ld + i];
    if (!dense::cholesky(k, L.data(), k)) return false;
    dense::chol_solve(k, L.data(), k, b.Vw.data(), k, pl);
    return true;
}

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

namespace rksm {

// The lock-step driver.  probs: distinct handles of box heat problems (2D or
// 3D, at least 3 points a side); each is solved exactly as solve_impl would,
// with every device step grouped over the batch on stream s.
int solve_batch_impl(int count, st_problem* const* probs, const double* const* F1, const int* ldf1,
                     const double* const* F2, const int* ldf2, const int* ncols, st_solution* sols, st_stats* stats,
                     int* status, cudaStream_t s, st_batch_stats* bs, int host_threads) {
    const auto T0 = Clock::now();
    st_batch_stats BS{};
    BS.instances = count;
    hostpar::ActiveSolve active;
    std::vector<BI> B(count);
    for (int i = 0; i < count; ++i) {
        BI& b = B[i];
        b.p = probs[i];
        b.own_stream = b.p->stream;
        b.p->stream = s;
        b.n = b.p->n_h;
        b.nt = b.p->n_t;
        b.c = Ctx{b.p, s, b.n};
        b.prec = b.p->d.precision;
        b.df = b.prec == ST_MIXED;
        b.dt = b.p->dt;
        b.tol = b.p->d.tol;
        b.F1 = F1[i];
        b.F2 = F2[i];
        b.ldf1 = ldf1[i];
        b.ldf2 = ldf2[i];
        b.p0 = ncols[i];
        b.sol = sols ? &sols[i] : nullptr;
        b.t0 = T0;
    }
    // the handles return to their own streams whatever happens below
    struct Restore {
        std::vector<BI>& B;
        ~Restore() {
            for (BI& b : B) b.p->stream = b.own_stream;
        }
    } restore{B};
    const int hw = std::max(1, (int)std::thread::hardware_concurrency());
    hostpar::Pool pool(std::max(1, std::min({host_threads, hw, count})));
    stg::GroupArena arena;
    BStage sg;
    int launches = 0;
    auto live_list = [&]() {
        std::vector<int> v;
        for (int i = 0; i < count; ++i)
            if (B[i].live) v.push_back(i);
        return v;
    };
    // ends a phase: launches issued, results downloaded, stream idle
    auto finish = [&](stg::GroupPhase& ph) -> int {
        ST_TRY(ph.run());
        launches += ph.launches();
        ST_TRY(sg.fetch(s));
        arena.reset();
        return ST_OK;
    };
    auto tick = [](Clock::time_point& t, double& acc) {
        const auto now = Clock::now();
        acc += ms_between(t, now);
        t = now;
    };
    auto tp = Clock::now();

    // ---- A1: rank compression of F = F1 F2^T ----
    {
        size_t need = 0;
        for (BI& b : B)
            need += pad32((size_t)b.p0 * b.p0) + (st_is_device_ptr(b.F2) ? pad32((size_t)b.nt * b.p0) : 0);
        ST_TRY(sg.reserve(need, s));
        stg::GroupPhase ph(s, &arena);
        std::vector<stg::TnTask> tn;
        for (BI& b : B) {
            double* part;
            ST_TRY(slot(b.p, S_F1D, (size_t)b.n * b.p0, &b.F1d));
            ST_TRY(st_stage_matrix(b.p, b.F1, b.ldf1, b.n, b.p0, b.F1d));
            ST_TRY(slot(b.p, S_PART, tn_part_elems(b.n, b.p0, b.p0), &part));
            b.dGF = sg.out((size_t)b.p0 * b.p0);
            tn_tasks(b.n, b.p0, b.p0, b.F1d, b.n, b.F1d, b.n, false, part, b.dGF, b.p0, tn);
            if (st_is_device_ptr(b.F2)) {
                b.dF2 = sg.out((size_t)b.nt * b.p0);
                ST_CUDA_TRY(cudaMemcpy2DAsync(b.dF2, sizeof(double) * b.nt, b.F2, sizeof(double) * b.ldf2,
                                              sizeof(double) * b.nt, b.p0, cudaMemcpyDeviceToDevice, s));
            }
        }
        ph.tn(false, tn);
        ST_TRY(finish(ph));
        pool.run(count, [&](int i) { compress_plan(B[i], sg.host_of(B[i].dGF)); });
        // an ill-conditioned F1 takes the column-wise QR (synchronous, per instance)
        for (BI& b : B)
            if (b.live && !b.gram && b.r1 > 0) {
                const int rc = block_qr(b.c, b.F1d, b.n, b.p0, 0.0, 1e-14, b.R1, &b.r1);
                if (rc != ST_OK) {
                    b.fail(rc);
                    continue;
                }
                b.T1.assign((size_t)b.r1 * b.r1, 0.0);
                for (int t = 0; t < b.r1; ++t) b.T1[(size_t)t * b.r1 + t] = 1.0;
                b.src_cols = b.r1;
            }
        std::vector<std::vector<double>> Tc(count);
        pool.run(count, [&](int i) {
            if (B[i].live) compress_finish(B[i], Tc[i]);
        });
        // F = 0: U = 0
        for (BI& b : B)
            if (b.live && b.r == 0) {
                b.k = 0;
                b.p->k = 0;
                if (b.sol) {
                    b.sol->n_h = b.n;
                    b.sol->n_t = b.nt;
                    b.sol->k = 0;
                    b.sol->V = b.p->V;
                    b.sol->Y = b.p->Y;
                    if (b.sol->U_dense)
                        for (int l = 0; l < b.nt; ++l)
                            ST_CUDA_TRY(cudaMemsetAsync(b.sol->U_dense + (size_t)l * b.sol->ldu, 0,
                                                        sizeof(double) * b.n, s));
                }
                b.S.converged = 1;
                b.status = ST_OK;
                b.live = false;
                b.res = 0.0;
            }
        tick(tp, BS.ms_phase[0]);

        // ---- start block: V = orth(M^{-1} F1c) ----
        need = 0;
        for (BI& b : B)
            if (b.live) need += pad32((size_t)b.r * b.r) + pad32(Tc[&b - &B[0]].size());
        ST_TRY(sg.reserve(need, s));
        SolveLaunches L;
        std::vector<stg::NnTask> nn;
        std::vector<stg::TnTask> tg;
        for (int i = 0; i < count; ++i) {
            BI& b = B[i];
            if (!b.live) continue;
            const int n = b.n, r = b.r;
            b.pmax = r;
            ST_TRY(slot(b.p, S_F1C, (size_t)n * r, &b.F1c));
            const double* dTc = sg.in(Tc[i].data(), Tc[i].size());
            nn_tasks(n, b.src_cols, r, 1.0, b.F1d, n, dTc, b.src_cols, 0.0, b.F1c, n, nn);
            ST_TRY(ensure_basis(b.p, b.c, std::min(2 * b.pmax + 8, b.p->d.max_basis + 16), 0, &b.MV));
            ST_TRY(slot(b.p, S_MAQ, (size_t)n * kNmaq * b.pmax, &b.MAq));
            const size_t nm = (size_t)n * r;
            double* V = b.p->V;
            if (b.prec == ST_FP64) {
                double* tmp;
                ST_TRY(slot(b.p, S_TMP, nm, &tmp));
                L.fd64.add<double>(b.p, FD_MASS_INVERSE, 0.0, 1.0, b.F1c, n, r, V, n, tmp);
            } else {
                float *x32, *w32, *t32;
                ST_TRY(slot(b.p, S_X32, nm, &x32));
                ST_TRY(slot(b.p, S_W32, nm, &w32));
                ST_TRY(slot(b.p, S_T32, nm, &t32));
                L.to32a.push_back(elem(stg::E_TO32, n, r, b.F1c, n, x32, n));
                L.fd32a.add<float>(b.p, FD_MASS_INVERSE, 0.0, 1.0, x32, n, r, w32, n, t32);
                L.add32a.push_back(elem(stg::E_ADD32, n, r, w32, n, V, n, 0.0, 0.0));
            }
            double* part;
            ST_TRY(slot(b.p, S_PART, tn_part_elems(n, r, r), &part));
            b.dG = sg.out((size_t)r * r);
            tn_tasks(n, r, r, V, n, V, n, false, part, b.dG, r, tg);
        }
        ST_TRY(sg.push(s));
        stg::GroupPhase ps(s, &arena);
        ps.nn(false, nn);
        L.issue(ps);
        // mixed: two refinement steps W += M^{-1} (X - M W), each with an FP32 transform
        for (int rep = 0; rep < 2; ++rep) {
            std::vector<stg::StencilTask> cm[4];
            std::vector<stg::ElemTask> ax, t32, a32;
            FdBatch fd(4);
            for (BI& b : B) {
                if (!b.live || b.prec == ST_FP64) continue;
                const int n = b.n, r = b.r;
                float *x32, *w32, *tt;
                double* r64;
                ST_TRY(slot(b.p, S_X32, (size_t)n * r, &x32));
                ST_TRY(slot(b.p, S_W32, (size_t)n * r, &w32));
                ST_TRY(slot(b.p, S_T32, (size_t)n * r, &tt));
                ST_TRY(slot(b.p, S_TMP, (size_t)n * r, &r64));
                cm[b.p->dim].push_back(comb_task(b.p, -1.0, 0.0, b.p->V, n, r, 0.0, r64, n));
                ax.push_back(elem(stg::E_AXPBY, n, r, b.F1c, n, r64, n, 1.0, 1.0));
                t32.push_back(elem(stg::E_TO32, n, r, r64, n, x32, n));
                fd.add<float>(b.p, FD_MASS_INVERSE, 0.0, 1.0, x32, n, r, w32, n, tt);
                a32.push_back(elem(stg::E_ADD32, n, r, w32, n, b.p->V, n, 0.0, 1.0));
            }
            ps.stencil(2, cm[2]);
            ps.stencil(3, cm[3]);
            ps.elem(ax);
            ps.elem(t32);
            fd.issue(ps);
            ps.elem(a32);
        }
        ps.tn(false, tg);
        ST_TRY(finish(ps));
        tick(tp, BS.ms_phase[1]);

        // first block QR, then the products of the start block
        pool.run(count, [&](int i) {
            BI& b = B[i];
            if (!b.live) return;
            qr_plan(sg.host_of(b.dG), b.r, 0.0, 1e-12, b.qp);
            if (b.qp.rank == 0) {
                breakdown("start block has rank 0");
                b.fail(ST_EBREAKDOWN);
            }
        });
        for (BI& b : B) {
            if (!b.live) continue;
            if (b.qp.fast) {
                b.k = b.r;
            } else {
                std::vector<double> Rx;
                const int rc = block_qr(b.c, b.p->V, b.n, b.r, 0.0, 1e-12, Rx, &b.k);
                if (rc != ST_OK) {
                    b.fail(rc);
                } else if (b.k == 0) {
                    breakdown("start block has rank 0");
                    b.fail(ST_EBREAKDOWN);
                }
            }
        }
        need = 0;
        for (BI& b : B)
            if (b.live)
                need += 3 * pad32((size_t)b.r * b.r) + pad32(1) + pad32((size_t)b.k * 2 * b.k) + pad32((size_t)b.k * b.r);
        ST_TRY(sg.reserve(need, s));
        std::vector<stg::TrsmTask> tr1, tr2;
        std::vector<stg::TnTask> tn2, tx0, tg1;
        std::vector<stg::CholTask> ch;
        std::vector<stg::ElemTask> todf, cpmv;
        std::vector<stg::StencilTask> ma[4];
        for (BI& b : B) {
            if (!b.live) continue;
            const int n = b.n, k = b.k, r = b.r;
            double* V = b.p->V;
            double* part;
            ST_TRY(slot(b.p, S_PART, std::max(tn_part_elems(n, k, 2 * k), tn_part_elems(n, k, r)), &part));
            b.dflag = nullptr;
            if (b.qp.fast) {
                const double* dR1 = sg.in(b.qp.R1.data(), (size_t)r * r);
                tr1.push_back(stg::TrsmTask{n, r, dR1, r, V, n});
                double* dG2 = sg.out((size_t)r * r);
                tn_tasks(n, r, r, V, n, V, n, false, part, dG2, r, tn2);
                b.dR2 = sg.out((size_t)r * r);
                b.dflag = sg.out(1);
                ch.push_back(stg::CholTask{r, dG2, r, b.dR2, r, b.dflag});
                tr2.push_back(stg::TrsmTask{n, r, b.dR2, r, V, n});
            }
            if (b.df) todf.push_back(elem(stg::E_TO_DF, n, k, V, n, b.p->Vdf, n));
            ma[b.p->dim].push_back(ma_task(b.p, V, n, k, b.MAq, b.MAq + (size_t)n * k, n));
            b.dX12 = sg.out((size_t)k * 2 * k);
            tn_tasks(n, k, 2 * k, V, n, b.MAq, n, false, part, b.dX12, k, tx0);
            b.dX3 = sg.out((size_t)k * r);
            cpmv.push_back(elem(stg::E_COPY64, n, k, b.MAq, n, b.MV, n));
        }
        ST_TRY(sg.push(s));
        stg::GroupPhase pb(s, &arena);
        pb.trsm(tr1);
        pb.tn(false, tn2);
        pb.chol(ch);
        pb.trsm(tr2);
        pb.elem(todf);
        pb.stencil(2, ma[2]);
        pb.stencil(3, ma[3]);
        pb.tn(false, tx0);
        // V^T F1c: its own launch (the partial room is shared with the product above)
        for (BI& b : B) {
            if (!b.live) continue;
            double* part = (double*)b.p->slot_ptr[S_PART];
            tn_tasks(b.n, b.k, b.r, b.p->V, b.n, b.F1c, b.n, false, part, b.dX3, b.k, tg1);
        }
        pb.tn(false, tg1);
        pb.elem(cpmv);
        ST_TRY(finish(pb));
        pool.run(count, [&](int i) {
            BI& b = B[i];
            if (!b.live) return;
            if (b.dflag && sg.host_of(b.dflag)[0] != 0.0) {
                breakdown("start block: device Cholesky pivot not positive");
                b.fail(ST_EBREAKDOWN);
                return;
            }
            const int k = b.k, r = b.r;
            const double* X = sg.host_of(b.dX12);
            const double* G = sg.host_of(b.dX3);
            b.Mm.grow(k);
            b.Am.grow(k);
            for (int j = 0; j < k; ++j)
                for (int q = 0; q < k; ++q) {
                    b.Mm(q, j) = 0.5 * (X[(size_t)j * k + q] + X[(size_t)q * k + j]);
                    b.Am(q, j) = 0.5 * (X[(size_t)(k + j) * k + q] + X[(size_t)(k + q) * k + j]);
                }
            b.ldg = std::max(64, 2 * k);
            b.Gm.assign((size_t)b.ldg * r, 0.0);
            for (int j = 0; j < r; ++j)
                for (int q = 0; q < k; ++q) b.Gm[(size_t)j * b.ldg + q] = G[(size_t)j * k + q];
            b.boff = {0};
            b.bsz = {k};
        });
        tick(tp, BS.ms_phase[3]);
    }

    // ---- rational Krylov iterations in lock step ----
    std::vector<int> act;
    while (true) {
        // loop-top exits of solve_impl, basis growth (allocations on the stream, in order)
        for (BI& b : B) {
            if (!b.live) continue;
            b.pl = b.bsz.back();
            b.lo = b.boff.back();
            if (b.it >= b.p->d.maxit || b.k + b.pl > b.p->d.max_basis) {
                b.live = false;   // status stays ST_ENOTCONV unless a check converged
                continue;
            }
            const int rc = ensure_basis(b.p, b.c, b.k + b.pl, b.k, &b.MV);
            if (rc != ST_OK) b.fail(rc);
        }
        act = live_list();
        if (act.empty()) break;
        ++BS.rounds;
        // shifts (host)
        pool.run((int)act.size(), [&](int j) {
            BI& b = B[act[j]];
            const auto t0 = Clock::now();
            const int k = b.k;
            if (b.last_ritz_k < 0 || k <= 16 ||
                k >= b.last_ritz_k + std::max(2, b.last_ritz_k / (b.last_ritz_k > 64 ? 4 : 8))) {
                if (!ritz_values(k, b.Am.a.data(), b.Mm.a.data(), b.Mm.ld, b.ritz)) b.ritz.clear();
                b.last_ritz_k = k;
            }
            b.s = next_shift(b.p->lam_min, b.p->lam_max, b.shifts, b.ritz, 80);
            b.shifts.push_back(b.s);
            ++b.it;
            b.S.ms_phase[7] += ms_between(t0, Clock::now());
        });
        tick(tp, BS.ms_phase[7]);

        // ---- phase A: shifted solve into the next basis slot, block CGS2 ----
        size_t need = 0;
        for (int i : act) need += 2 * pad32((size_t)(B[i].k + B[i].pl) * B[i].pl);
        ST_TRY(sg.reserve(need, s));
        SolveLaunches L;
        std::vector<stg::ElemTask> tdf[2];
        std::vector<stg::TnTask> tn_df[2], tn_64[2];
        std::vector<stg::NnTask> nn_df[2], nn_64[2];
        for (int i : act) {
            BI& b = B[i];
            const int n = b.n, k = b.k, pl = b.pl;
            b.kk = k + pl;
            b.W = b.p->V + (size_t)k * n;
            ST_TRY(add_resolvent(b, b.s, b.p->V + (size_t)b.lo * n, b.MV + (size_t)b.lo * n, pl, b.W, L));
            double* part;
            ST_TRY(slot(b.p, S_PART, tn_part_elems(n, b.kk, pl), &part));
            for (int pass = 0; pass < 2; ++pass) {
                b.dh[pass] = sg.out((size_t)b.kk * pl);
                if (b.df) {
                    float2* Vdf = b.p->Vdf;
                    tdf[pass].push_back(elem(stg::E_TO_DF, n, pl, b.W, n, Vdf + (size_t)k * n, n));
                    tn_tasks(n, b.kk, pl, Vdf, n, Vdf + (size_t)k * n, n, true, part, b.dh[pass], b.kk, tn_df[pass]);
                    nn_tasks(n, k, pl, -1.0, Vdf, n, b.dh[pass], b.kk, 1.0, b.W, n, nn_df[pass]);
                } else {
                    tn_tasks(n, b.kk, pl, b.p->V, n, b.W, n, false, part, b.dh[pass], b.kk, tn_64[pass]);
                    nn_tasks(n, k, pl, -1.0, b.p->V, n, b.dh[pass], b.kk, 1.0, b.W, n, nn_64[pass]);
                }
            }
        }
        stg::GroupPhase pa(s, &arena);
        L.issue(pa);
        for (int pass = 0; pass < 2; ++pass) {
            pa.elem(tdf[pass]);
            pa.tn(true, tn_df[pass], pass == 0);   // first pass: FP32 on the leading parts
            pa.tn(false, tn_64[pass]);
            pa.nn(true, nn_df[pass]);
            pa.nn(false, nn_64[pass]);
        }
        ST_TRY(finish(pa));
        tick(tp, BS.ms_phase[1]);

        // ---- host: Gram matrix of the new block -> rank and first CholQR factor ----
        pool.run((int)act.size(), [&](int j) {
            BI& b = B[act[j]];
            const int k = b.k, pl = b.pl, kk = b.kk;
            b.Hcol.assign((size_t)k * pl, 0.0);
            b.Gw.assign((size_t)pl * pl, 0.0);
            double tr1 = 0.0, tr2 = 0.0;
            b.ref2 = 0.0;
            const double* h0 = sg.host_of(b.dh[0]);
            const double* h1 = sg.host_of(b.dh[1]);
            for (int c = 0; c < pl; ++c)
                for (int q = 0; q < k; ++q) b.Hcol[(size_t)c * k + q] = h0[(size_t)c * kk + q] + h1[(size_t)c * kk + q];
            for (int c = 0; c < pl; ++c) {
                b.ref2 = std::max(b.ref2, h0[(size_t)c * kk + k + c]);
                for (int q = 0; q < pl; ++q) {
                    const double g = h1[(size_t)c * kk + k + q];
                    double hh = 0.0;
                    for (int t = 0; t < k; ++t) hh += h1[(size_t)q * kk + t] * h1[(size_t)c * kk + t];
                    b.Gw[(size_t)c * pl + q] = g - hh;
                    if (q == c) {
                        tr1 += g;
                        tr2 += hh;
                    }
                }
            }
            b.explicit_gram = !(tr2 <= 1e-4 * tr1);
            if (!b.explicit_gram) qr_plan(b.Gw.data(), pl, b.ref2, 1e-10, b.qp);
        });
        // rare blocks: explicit Gram matrix, a third FP64 pass, the column-wise QR (per instance)
        for (int i : act) {
            BI& b = B[i];
            const int n = b.n, k = b.k, pl = b.pl;
            int rc = ST_OK;
            if (b.explicit_gram) {
                rc = ts_tn_host(b.c, pl, pl, b.W, n, b.W, n, b.Gw.data());
                if (rc == ST_OK) qr_plan(b.Gw.data(), pl, b.ref2, 1e-10, b.qp);
            }
            if (rc == ST_OK && b.qp.severe) {
                std::vector<double> h3((size_t)k * pl), G3((size_t)pl * pl);
                rc = ts_tn_host(b.c, k, pl, b.p->V, n, b.W, n, h3.data());
                if (rc == ST_OK) rc = ts_nn_host(b.c, k, pl, -1.0, b.p->V, n, h3.data(), 1.0, b.W, n);
                if (rc == ST_OK) {
                    for (size_t q = 0; q < b.Hcol.size(); ++q) b.Hcol[q] += h3[q];
                    rc = ts_tn_host(b.c, pl, pl, b.W, n, b.W, n, G3.data());
                }
                if (rc == ST_OK) qr_plan(G3.data(), pl, b.ref2, 1e-10, b.qp);
            }
            b.pn = 0;
            b.Rq.assign((size_t)pl * pl, 0.0);
            if (rc == ST_OK && b.qp.rank > 0) {
                if (b.qp.fast)
                    b.pn = pl;
                else
                    rc = block_qr(b.c, b.W, n, pl, b.ref2, 1e-10, b.Rq, &b.pn);
            }
            if (rc != ST_OK) b.fail(rc);
        }
        tick(tp, BS.ms_phase[2]);

        // ---- phase B: CholQR2 on the device, products of the new block ----
        need = 0;
        for (int i : act) {
            const BI& b = B[i];
            if (!b.live || b.pn == 0) continue;
            const int kq = b.k + b.pn;
            need += 3 * pad32((size_t)b.pl * b.pl) + pad32(1) + pad32((size_t)kq * kNmaq * b.pn) +
                    pad32((size_t)b.pn * b.r);
        }
        ST_TRY(sg.reserve(need, s));
        std::vector<stg::TrsmTask> tr1, tr2;
        std::vector<stg::TnTask> tg2, tx_df, tx_64, tx3;
        std::vector<stg::CholTask> ch;
        std::vector<stg::ElemTask> todf;
        std::vector<stg::StencilTask> ma[4];
        for (int i : act) {
            BI& b = B[i];
            b.dflag = nullptr;
            if (!b.live || b.pn == 0) continue;
            const int n = b.n, k = b.k, pl = b.pl, pn = b.pn, kq = k + pn;
            double* part;
            ST_TRY(slot(b.p, S_PART,
                        std::max({tn_part_elems(n, pl, pl), tn_part_elems(n, kq, kNmaq * pn), tn_part_elems(n, pn, b.r)}),
                        &part));
            if (b.qp.fast) {
                const double* dR1 = sg.in(b.qp.R1.data(), (size_t)pl * pl);
                tr1.push_back(stg::TrsmTask{n, pl, dR1, pl, b.W, n});
                double* dG2 = sg.out((size_t)pl * pl);
                tn_tasks(n, pl, pl, b.W, n, b.W, n, false, part, dG2, pl, tg2);
                b.dR2 = sg.out((size_t)pl * pl);
                b.dflag = sg.out(1);
                ch.push_back(stg::CholTask{pl, dG2, pl, b.dR2, pl, b.dflag});
                tr2.push_back(stg::TrsmTask{n, pl, b.dR2, pl, b.W, n});
            }
            ma[b.p->dim].push_back(ma_task(b.p, b.W, n, pn, b.MAq, b.MAq + (size_t)n * pn, n));
            b.dX12 = sg.out((size_t)kq * kNmaq * pn);
            if (b.df) {
                float2* W2;
                ST_TRY(slot(b.p, S_WDF, (size_t)n * kNmaq * pn, &W2));
                todf.push_back(elem(stg::E_TO_DF, n, pn, b.W, n, b.p->Vdf + (size_t)k * n, n));
                todf.push_back(elem(stg::E_TO_DF, n, kNmaq * pn, b.MAq, n, W2, n));
                tn_tasks(n, kq, kNmaq * pn, b.p->Vdf, n, W2, n, true, part, b.dX12, kq, tx_df);
            } else {
                tn_tasks(n, kq, kNmaq * pn, b.p->V, n, b.MAq, n, false, part, b.dX12, kq, tx_64);
            }
            b.dX3 = sg.out((size_t)pn * b.r);
            tn_tasks(n, pn, b.r, b.W, n, b.F1c, n, false, part, b.dX3, pn, tx3);
        }
        ST_TRY(sg.push(s));
        stg::GroupPhase pb(s, &arena);
        pb.trsm(tr1);
        pb.tn(false, tg2);
        pb.chol(ch);
        pb.trsm(tr2);
        pb.stencil(2, ma[2]);
        pb.stencil(3, ma[3]);
        pb.elem(todf);
        pb.tn(true, tx_df);
        pb.tn(false, tx_64);
        pb.tn(false, tx3);
        ST_TRY(finish(pb));
        pool.run((int)act.size(), [&](int j) {
            BI& b = B[act[j]];
            if (!b.live) return;
            const int k = b.k, pl = b.pl, pn = b.pn, kq = k + pn;
            if (pn > 0) {
                if (b.qp.fast) {
                    if (sg.host_of(b.dflag)[0] != 0.0) {
                        breakdown("new block: device Cholesky pivot not positive");
                        b.fail(ST_EBREAKDOWN);
                        return;
                    }
                    b.Rq = upper_product(pl, sg.host_of(b.dR2), b.qp.R1.data());
                }
                const double* x12 = sg.host_of(b.dX12);
                b.X1.resize((size_t)k * kNmaq * pn);
                b.X2.resize((size_t)pn * 2 * pn);
                for (int c = 0; c < kNmaq * pn; ++c)
                    for (int q = 0; q < k; ++q) b.X1[(size_t)c * k + q] = x12[(size_t)c * kq + q];
                for (int c = 0; c < 2 * pn; ++c)
                    for (int q = 0; q < pn; ++q) b.X2[(size_t)c * pn + q] = x12[(size_t)c * kq + k + q];
                b.X3.assign(sg.host_of(b.dX3), sg.host_of(b.dX3) + (size_t)pn * b.r);
            }
            b.mu_extra = pn;
            b.Hb.grow(k + pn);
            for (int c = 0; c < pl; ++c) {
                for (int q = 0; q < k; ++q) b.Hb(q, b.lo + c) = b.Hcol[(size_t)c * k + q];
                for (int q = 0; q < pn; ++q) b.Hb(k + q, b.lo + c) = b.Rq[(size_t)c * pl + q];
            }
            b.check = pn == 0 || b.it >= b.next_check || b.it >= b.p->d.maxit || k + pn + pn > b.p->d.max_basis;
            if (b.check && pn > 0 && !residual_inputs(b)) {
                breakdown("residual: projected mass matrix not positive definite");
                b.fail(ST_EBREAKDOWN);
            }
        });
        tick(tp, BS.ms_phase[3]);

        // ---- phase C (checks): residual direction's Gram matrix on the device while the
        // host solves the projected equations ----
        need = 0;
        for (int i : act) {
            const BI& b = B[i];
            if (b.live && b.check && b.pn > 0)
                need += pad32((size_t)b.pn * b.pl) + pad32((size_t)b.k * b.pl) + pad32((size_t)b.pl * b.pl);
        }
        ST_TRY(sg.reserve(need, s));
        std::vector<stg::ElemTask> ccopy, caxpy;
        std::vector<stg::NnTask> cn1, cn2;
        std::vector<stg::TnTask> ctn;
        for (int i : act) {
            BI& b = B[i];
            b.dGb = nullptr;
            if (!b.live || !b.check || b.pn == 0) continue;
            const int n = b.n, k = b.k, pn = b.pn, pl = b.pl;
            double *Wh, *Wh2, *part;
            ST_TRY(slot(b.p, S_WH, (size_t)n * pl, &Wh));
            ST_TRY(slot(b.p, S_WH2, (size_t)n * pl, &Wh2));
            ST_TRY(slot(b.p, S_PART, std::max(tn_part_elems(n, pl, pl), (size_t)1), &part));
            ccopy.push_back(elem(stg::E_COPY64, n, pn, b.MAq + (size_t)n * pn, n, Wh, n));
            caxpy.push_back(elem(stg::E_AXPBY, n, pn, b.MAq, n, Wh, n, b.s, 1.0));
            const double* dnr = sg.in(b.negR.data(), b.negR.size());
            nn_tasks(n, pn, pl, 1.0, Wh, n, dnr, pn, 0.0, Wh2, n, cn1);
            const double* dvw = sg.in(b.Vw.data(), b.Vw.size());
            nn_tasks(n, k, pl, -1.0, b.MV, n, dvw, k, 1.0, Wh2, n, cn2);
            b.dGb = sg.out((size_t)pl * pl);
            tn_tasks(n, pl, pl, Wh2, n, Wh2, n, false, part, b.dGb, pl, ctn);
        }
        bool any_check = false;
        for (int i : act) any_check = any_check || (B[i].live && B[i].check);
        if (any_check) {
            ST_TRY(sg.push(s));
            stg::GroupPhase pc(s, &arena);
            pc.elem(ccopy);
            pc.elem(caxpy);
            pc.nn(false, cn1);
            pc.nn(false, cn2);
            pc.tn(false, ctn);
            ST_TRY(pc.run());
            launches += pc.launches();
            // the projected equations of the checking instances, while the device works; the
            // costliest first, each with its share of the host threads
            std::vector<int> chk;
            for (int i : act)
                if (B[i].live && B[i].check) chk.push_back(i);
            std::stable_sort(chk.begin(), chk.end(), [&](int a, int b) {
                return (double)B[a].k * B[a].k * B[a].nt > (double)B[b].k * B[b].k * B[b].nt;
            });
            pool.run((int)chk.size(), [&](int j) {
                BI& b = B[chk[j]];
                const auto t0 = Clock::now();
                if (!projected_solve(b.k, b.nt, b.dt, b.Mm.a.data(), b.Am.a.data(), b.Mm.ld, b.Gm.data(), b.ldg, b.r,
                                     b.F2c.data(), b.Y, true)) {
                    breakdown("projected equation singular");
                    b.fail(ST_EBREAKDOWN);
                }
                b.S.residual_checks++;
                b.S.ms_phase[4] += ms_between(t0, Clock::now());
            });
            tick(tp, BS.ms_phase[4]);
            ST_TRY(sg.fetch(s));
            arena.reset();
            pool.run((int)act.size(), [&](int j) {
                BI& b = B[act[j]];
                if (!b.live || !b.check) return;
                const auto t0 = Clock::now();
                double rr = 0.0;
                if (b.pn > 0) {
                    bool ok = true;
                    rr = residual_norm2(b, sg.host_of(b.dGb), &ok);
                    if (!ok) {
                        breakdown("rational Arnoldi Hessenberg matrix singular");
                        b.fail(ST_EBREAKDOWN);
                        return;
                    }
                }
                b.res = std::sqrt(std::max(rr, 0.0)) / b.normF;
                b.S.ms_phase[5] += ms_between(t0, Clock::now());
                if (b.res <= b.tol || b.pn == 0) {
                    b.status = b.res <= b.tol ? ST_OK : ST_ENOTCONV;
                    if (b.pn == 0 && b.res > b.tol) b.status = ST_EBREAKDOWN;
                    b.live = false;
                    return;
                }
                b.next_check = b.it + check_gap(b.hist_it, b.hist_res, b.it, b.res, b.tol, (double)b.k * b.k * b.nt);
                b.hist_it.push_back(b.it);
                b.hist_res.push_back(b.res);
            });
            tick(tp, BS.ms_phase[5]);
        }

        // ---- append the new blocks ----
        std::vector<stg::ElemTask> app;
        for (int i : act) {
            BI& b = B[i];
            if (!b.live) continue;
            if (b.pn == 0) {
                b.status = ST_EBREAKDOWN;
                b.live = false;
                continue;
            }
            app.push_back(elem(stg::E_COPY64, b.n, b.pn, b.MAq, b.n, b.MV + (size_t)b.k * b.n, b.n));
        }
        if (!app.empty()) {
            stg::GroupPhase pm(s, &arena);   // ordered before the next growth of the bases
            pm.elem(app);
            ST_TRY(pm.run());
            launches += pm.launches();
        }
        pool.run((int)act.size(), [&](int j) {
            BI& b = B[act[j]];
            if (!b.live) return;
            const int k = b.k, pn = b.pn, kn = k + pn;
            b.Mm.grow(kn);
            b.Am.grow(kn);
            for (int c = 0; c < pn; ++c) {
                for (int q = 0; q < k; ++q) {
                    b.Mm(q, k + c) = b.Mm(k + c, q) = b.X1[(size_t)c * k + q];
                    b.Am(q, k + c) = b.X1[(size_t)(pn + c) * k + q];
                    b.Am(k + c, q) = b.X1[(size_t)(pn + c) * k + q];
                }
                for (int q = 0; q < pn; ++q) {
                    b.Mm(k + q, k + c) = 0.5 * (b.X2[(size_t)c * pn + q] + b.X2[(size_t)q * pn + c]);
                    b.Am(k + q, k + c) = 0.5 * (b.X2[(size_t)(pn + c) * pn + q] + b.X2[(size_t)(pn + q) * pn + c]);
                }
            }
            if (kn > b.ldg) {
                const int nl = std::max(2 * b.ldg, kn);
                std::vector<double> g2((size_t)nl * b.r, 0.0);
                for (int c = 0; c < b.r; ++c)
                    for (int q = 0; q < k; ++q) g2[(size_t)c * nl + q] = b.Gm[(size_t)c * b.ldg + q];
                b.Gm.swap(g2);
                b.ldg = nl;
            }
            for (int c = 0; c < b.r; ++c)
                for (int q = 0; q < pn; ++q) b.Gm[(size_t)c * b.ldg + k + q] = b.X3[(size_t)c * pn + q];
            b.boff.push_back(k);
            b.bsz.push_back(pn);
            b.k = kn;
        });
        tick(tp, BS.ms_phase[3]);
    }

    // ---- A9 output ----
    pool.run(count, [&](int i) {
        BI& b = B[i];
        if (b.r == 0 || b.k == 0 || b.aborted) return;
        if (b.Y.empty() || (int)(b.Y.size() / std::max(1, b.nt)) != b.k) {
            if (!projected_solve(b.k, b.nt, b.dt, b.Mm.a.data(), b.Am.a.data(), b.Mm.ld, b.Gm.data(), b.ldg, b.r,
                                 b.F2c.data(), b.Y, true)) {
                breakdown("projected equation singular (final basis)");
                b.status = ST_EBREAKDOWN;
                b.Y.clear();
                return;
            }
            b.mu_extra = 0;
        }
    });
    int rc_all = ST_OK;
    for (BI& b : B) {
        if (b.r == 0 || b.k == 0 || b.aborted || b.Y.empty()) continue;
        st_problem* p = b.p;
        const int k = b.k, nt = b.nt;
        if (p->Y_cap < (size_t)k * nt) {
            if (p->Y) st_free_one(p, p->Y);
            p->Y = nullptr;
            p->Y_cap = 0;
            const int rc = st_alloc(p, (void**)&p->Y, sizeof(double) * (size_t)k * nt);
            if (rc != ST_OK) {
                b.status = rc;
                continue;
            }
            p->Y_cap = (size_t)k * nt;
        }
        ST_TRY(write_dev(b.c, b.Y.data(), k, k, nt, p->Y, k));
        p->k = k;
        if (b.sol) {
            b.sol->n_h = b.n;
            b.sol->n_t = nt;
            b.sol->k = k;
            b.sol->V = p->V;
            b.sol->Y = p->Y;
            if (b.sol->U_dense) {
                if (b.sol->ldu < b.n) {
                    b.status = ST_EINVAL;
                    continue;
                }
                ST_TRY(st_lowrank_dense(b.n, k, nt, p->V, b.n, p->Y, k, b.sol->U_dense, b.sol->ldu, s));
            }
        }
    }
    ST_CUDA_TRY(cudaStreamSynchronize(s));
    tick(tp, BS.ms_phase[6]);
    pool.run(count, [&](int i) {
        BI& b = B[i];
        st_stats& S = b.S;
        if (b.aborted) return;
        const int k = b.k, nt = b.nt;
        if (k > 0 && !b.Y.empty()) {
            std::vector<double> G((size_t)k * k, 0.0), w(k);
            for (int l = 0; l < nt; ++l) {
                const double* y = &b.Y[(size_t)l * k];
                for (int j = 0; j < k; ++j)
                    for (int q = 0; q <= j; ++q) G[(size_t)j * k + q] += y[q] * y[j];
            }
            for (int j = 0; j < k; ++j)
                for (int q = j + 1; q < k; ++q) G[(size_t)j * k + q] = G[(size_t)q * k + j];
            dense::sym_eigvals(k, G.data(), k, w.data());
            const double smax = std::sqrt(std::max(w[k - 1], 0.0));
            int rank = 0;
            for (int q = 0; q < k; ++q) rank += std::sqrt(std::max(w[q], 0.0)) > 1e-8 * smax;
            S.rank = rank;
        }
        S.iterations = b.it;
        S.basis_cols = k;
        S.mu_mem = k + b.mu_extra;
        S.relres = b.res;
        S.converged = b.res <= b.tol;
        if (!b.shifts.empty()) {
            S.shift_min = *std::min_element(b.shifts.begin(), b.shifts.end());
            S.shift_max = *std::max_element(b.shifts.begin(), b.shifts.end());
        }
        S.ms_total = ms_between(T0, Clock::now());
        if (b.status == ST_EBREAKDOWN && b.res <= b.tol) b.status = ST_OK;
    });
    for (int i = 0; i < count; ++i) {
        if (stats) stats[i] = B[i].S;
        if (status) status[i] = B[i].status;
    }
    BS.grouped_launches = launches;
    BS.ms_total = ms_between(T0, Clock::now());
    if (bs) *bs = BS;
    return rc_all;
}

}  // namespace rksm

// ---- C ABI ----
namespace {
// Problems the grouped path covers: box heat problems of 2 or 3 dimensions
// with at least 3 points a side (box stencils and fast diagonalisation).
bool groupable(const st_problem* p) {
    return p->tensor_heat && p->box_ok && (p->dim == 2 || p->dim == 3) && p->d.op == ST_HEAT;
}
}  // namespace

extern "C" int st_solve_batch(int count, st_problem* const* problems, const double* const* F1, const int* ldf1,
                              const double* const* F2, const int* ldf2, const int* ncols, st_solution* sols,
                              st_stats* stats, int* status, void* stream, int groups, st_batch_stats* bstats) {
    if (count < 0 || (count > 0 && (!problems || !F1 || !ldf1 || !F2 || !ldf2 || !ncols || !status))) return ST_EINVAL;
    if (bstats) *bstats = st_batch_stats{};
    if (count == 0) return ST_OK;
    int dev = 0;
    ST_CUDA_TRY(cudaGetDevice(&dev));
    std::vector<st_problem*> seen;
    for (int i = 0; i < count; ++i) {
        st_problem* p = problems[i];
        if (!p || !F1[i] || !F2[i] || ncols[i] < 1 || ncols[i] > 16 || ldf1[i] < p->n_h || ldf2[i] < p->n_t) {
            st_note_msg("st_solve_batch: bad problem, load pointer, leading dimension or column count");
            return ST_EINVAL;
        }
        if (p->device != dev) {
            st_note_msg("st_solve_batch: a problem belongs to another device than the current one");
            return ST_EINVAL;
        }
        seen.push_back(p);
    }
    std::sort(seen.begin(), seen.end());
    if (std::adjacent_find(seen.begin(), seen.end()) != seen.end()) {
        st_note_msg("st_solve_batch: the same problem handle appears twice");
        return ST_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int> grp, one;
    for (int i = 0; i < count; ++i) (groupable(problems[i]) ? grp : one).push_back(i);
    const auto t0 = Clock::now();
    st_batch_stats bs{};
    if (!grp.empty()) {
        const int m = (int)grp.size();
        std::vector<st_problem*> P(m);
        std::vector<const double*> f1(m), f2(m);
        std::vector<int> l1(m), l2(m), nc(m), stt(m, ST_OK);
        std::vector<st_solution> so(m);
        std::vector<st_stats> sst(m);
        for (int j = 0; j < m; ++j) {
            const int i = grp[j];
            P[j] = problems[i];
            f1[j] = F1[i];
            f2[j] = F2[i];
            l1[j] = ldf1[i];
            l2[j] = ldf2[i];
            nc[j] = ncols[i];
            if (sols) so[j] = sols[i];
        }
        // Lock-step groups on their own streams and host threads: while one group's host work runs (rank
        // decisions, shifts, projected solves), the others' grouped launches keep the device busy.  Problems
        // are dealt to the groups in decreasing order of size, so every group gets a share of the large ones.
        const int hw = std::max(1, (int)std::thread::hardware_concurrency());
        // automatic: groups of about 8 problems (measured on the 256-problem batch: 1 group 1.6 s, 4 groups
        // 1.19 s, 32 groups 0.97 s; lock step couples fast and slow problems, so small groups win)
        const int G = groups > 0 ? std::min(groups, m) : std::max(1, std::min(32, (m + 7) / 8));
        std::vector<int> order(m);
        for (int j = 0; j < m; ++j) order[j] = j;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            return (double)P[a]->n_h * P[a]->n_t > (double)P[b]->n_h * P[b]->n_t;
        });
        // (round robin measured faster than contiguous runs of similar problems, with or without stream
        // priorities favouring the costliest groups: 0.89-0.93 s against 1.04-1.14 s on the 256-problem batch)
        std::vector<std::vector<int>> members(G);
        for (int j = 0; j < m; ++j) members[j % G].push_back(order[j]);
        std::vector<int> rcs(G, ST_OK);
        const int per_group = std::max(1, std::min(16, hw) / G);   // host threads of each group's pool
        std::vector<st_batch_stats> gbs(G);
        auto run_group = [&](int g, cudaStream_t gs) {
            const std::vector<int>& mem = members[g];
            const int c = (int)mem.size();
            std::vector<st_problem*> Pg(c);
            std::vector<const double*> f1g(c), f2g(c);
            std::vector<int> l1g(c), l2g(c), ncg(c), stg_(c, ST_OK);
            std::vector<st_solution> sog(c);
            std::vector<st_stats> ssg(c);
            for (int q = 0; q < c; ++q) {
                const int j = mem[q];
                Pg[q] = P[j];
                f1g[q] = f1[j];
                f2g[q] = f2[j];
                l1g[q] = l1[j];
                l2g[q] = l2[j];
                ncg[q] = nc[j];
                sog[q] = so[j];
            }
            rcs[g] = solve_batch_impl(c, Pg.data(), f1g.data(), l1g.data(), f2g.data(), l2g.data(), ncg.data(),
                                      sols ? sog.data() : nullptr, ssg.data(), stg_.data(), gs, &gbs[g],
                                      per_group);
            for (int q = 0; q < c; ++q) {
                const int j = mem[q];
                stt[j] = stg_[q];
                sst[j] = ssg[q];
                so[j] = sog[q];
            }
        };
        if (G == 1) {
            run_group(0, s);
        } else {
            std::vector<cudaStream_t> gs(G, nullptr);
            cudaEvent_t start = nullptr;
            ST_CUDA_TRY(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
            ST_CUDA_TRY(cudaEventRecord(start, s));
            for (int g = 0; g < G; ++g) {
                ST_CUDA_TRY(cudaStreamCreateWithFlags(&gs[g], cudaStreamNonBlocking));
                ST_CUDA_TRY(cudaStreamWaitEvent(gs[g], start, 0));
            }
            std::vector<std::thread> th;
            for (int g = 1; g < G; ++g)
                th.emplace_back([&, g] {
                    cudaSetDevice(dev);
                    run_group(g, gs[g]);
                });
            run_group(0, gs[0]);
            for (auto& t : th) t.join();
            for (int g = 0; g < G; ++g) {
                cudaStreamSynchronize(gs[g]);
                cudaStreamDestroy(gs[g]);
            }
            cudaEventDestroy(start);
        }
        for (int g = 0; g < G; ++g) {
            if (rcs[g] != ST_OK) return rcs[g];
            bs.rounds = std::max(bs.rounds, gbs[g].rounds);
            bs.grouped_launches += gbs[g].grouped_launches;
            for (int q = 0; q < 8; ++q) bs.ms_phase[q] = std::max(bs.ms_phase[q], gbs[g].ms_phase[q]);
        }
        bs.groups = G;
        for (int j = 0; j < m; ++j) {
            const int i = grp[j];
            status[i] = stt[j];
            if (stats) stats[i] = sst[j];
            if (sols) sols[i] = so[j];
        }
    }
    // the rest one after another on the same stream, as st_solve
    for (int i : one) {
        st_problem* p = problems[i];
        cudaStream_t own = p->stream;
        p->stream = s;
        st_stats st{};
        status[i] = p->dim < 0 || (p->dim == 0 && p->d.op != ST_HEAT)
                        ? ST_ENOTSUP
                        : solve_impl(p, F1[i], ldf1[i], F2[i], ldf2[i], ncols[i], sols ? &sols[i] : nullptr, &st);
        p->stream = own;
        if (stats) stats[i] = st;
    }
    bs.instances = count;
    bs.grouped = (int)grp.size();
    bs.ms_total = ms_between(t0, Clock::now());
    if (bstats) *bstats = bs;
    return ST_OK;
}
