// P1 assembly on simplex meshes (paper Section 3: the conforming space X_h of
// continuous piecewise linear functions vanishing on the boundary), host side:
// the CSR input of a general-mesh problem.  See st_p1_mesh_csr in st.h.
#include <algorithm>
#include <cmath>
#include <vector>

#include "st.h"

namespace {

struct Entry {
    int r, c;
    double m, a;
};

// inverse and determinant of a d x d matrix (d = 2 or 3), row-major
bool invert(int d, const double* B, double* Bi, double* det) {
    if (d == 2) {
        const double dt = B[0] * B[3] - B[1] * B[2];
        if (dt == 0.0) return false;
        Bi[0] = B[3] / dt;
        Bi[1] = -B[1] / dt;
        Bi[2] = -B[2] / dt;
        Bi[3] = B[0] / dt;
        *det = dt;
        return true;
    }
    const double c00 = B[4] * B[8] - B[5] * B[7], c01 = B[5] * B[6] - B[3] * B[8], c02 = B[3] * B[7] - B[4] * B[6];
    const double dt = B[0] * c00 + B[1] * c01 + B[2] * c02;
    if (dt == 0.0) return false;
    // adjugate / det (Bi = B^-1, row-major)
    Bi[0] = c00 / dt;
    Bi[1] = (B[2] * B[7] - B[1] * B[8]) / dt;
    Bi[2] = (B[1] * B[5] - B[2] * B[4]) / dt;
    Bi[3] = c01 / dt;
    Bi[4] = (B[0] * B[8] - B[2] * B[6]) / dt;
    Bi[5] = (B[2] * B[3] - B[0] * B[5]) / dt;
    Bi[6] = c02 / dt;
    Bi[7] = (B[1] * B[6] - B[0] * B[7]) / dt;
    Bi[8] = (B[0] * B[4] - B[1] * B[3]) / dt;
    *det = dt;
    return true;
}

}  // namespace

extern "C" int st_p1_mesh_csr(int dim, int n_nodes, const double* xyz, int n_elems, const int* elems,
                              const unsigned char* interior, double kappa, int* row_ptr, int* col_idx,
                              double* m_vals, double* a_vals, int* n_h, int* nnz) {
    if ((dim != 2 && dim != 3) || n_nodes < 1 || n_elems < 1 || !xyz || !elems || !interior || !n_h || !nnz)
        return ST_EINVAL;
    const bool fill = row_ptr || col_idx || m_vals || a_vals;
    if (fill && !(row_ptr && col_idx && m_vals && a_vals)) return ST_EINVAL;
    std::vector<int> idx(n_nodes, -1);
    int nh = 0;
    for (int i = 0; i < n_nodes; ++i)
        if (interior[i]) idx[i] = nh++;
    const int nv = dim + 1;
    double fact = dim == 2 ? 2.0 : 6.0;
    std::vector<Entry> coo;
    coo.reserve((size_t)n_elems * nv * nv);
    for (int e = 0; e < n_elems; ++e) {
        const int* v = elems + (size_t)e * nv;
        for (int q = 0; q < nv; ++q)
            if (v[q] < 0 || v[q] >= n_nodes) return ST_EINVAL;
        double B[9], Bi[9], det = 0.0;
        // B[r][c] = x_{c+1}[r] - x_0[r] (columns are the edge vectors)
        for (int r = 0; r < dim; ++r)
            for (int c = 0; c < dim; ++c)
                B[r * dim + c] = xyz[(size_t)v[c + 1] * dim + r] - xyz[(size_t)v[0] * dim + r];
        if (!invert(dim, B, Bi, &det)) return ST_EINVAL;
        const double vol = std::fabs(det) / fact;
        // gradients: grad l_{i} = row i-1 of B^-1 (i = 1..d), grad l_0 = -sum
        double G[4][3] = {};
        for (int i = 1; i < nv; ++i)
            for (int k = 0; k < dim; ++k) G[i][k] = Bi[(i - 1) * dim + k];
        for (int k = 0; k < dim; ++k) {
            double s = 0.0;
            for (int i = 1; i < nv; ++i) s += G[i][k];
            G[0][k] = -s;
        }
        const double mdiag = 2.0 * vol / ((dim + 1) * (dim + 2)), moff = vol / ((dim + 1) * (dim + 2));
        for (int i = 0; i < nv; ++i) {
            const int ri = idx[v[i]];
            if (ri < 0) continue;
            for (int j = 0; j < nv; ++j) {
                const int cj = idx[v[j]];
                if (cj < 0) continue;
                double g = 0.0;
                for (int k = 0; k < dim; ++k) g += G[i][k] * G[j][k];
                coo.push_back({ri, cj, i == j ? mdiag : moff, kappa * vol * g});
            }
        }
    }
    std::stable_sort(coo.begin(), coo.end(), [](const Entry& a, const Entry& b) {
        return a.r != b.r ? a.r < b.r : a.c < b.c;
    });
    // merge duplicates (in element order within each (r, c)) and count
    int count = 0;
    for (size_t t = 0; t < coo.size(); ++t)
        if (t == 0 || coo[t].r != coo[t - 1].r || coo[t].c != coo[t - 1].c) ++count;
    *n_h = nh;
    *nnz = count;
    if (!fill) return ST_OK;
    int out = -1;
    for (int r = 0; r <= nh; ++r) row_ptr[r] = 0;
    for (size_t t = 0; t < coo.size(); ++t) {
        if (t == 0 || coo[t].r != coo[t - 1].r || coo[t].c != coo[t - 1].c) {
            ++out;
            col_idx[out] = coo[t].c;
            m_vals[out] = 0.0;
            a_vals[out] = 0.0;
            row_ptr[coo[t].r + 1]++;
        }
        m_vals[out] += coo[t].m;
        a_vals[out] += coo[t].a;
    }
    for (int r = 0; r < nh; ++r) row_ptr[r + 1] += row_ptr[r];
    return ST_OK;
}
