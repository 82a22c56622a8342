"""The executor's HBM admission estimate (st_request_bytes) on the CPU: a host-only call of the C ABI.

Checked against the footprint its header documents (operators, tables, basis, work columns, Y, flexible GMRES
blocks) and for the properties admission relies on: more unknowns, columns, mixed precision or a nonsymmetric
operator never lower the estimate, and max_basis caps the basis.
"""

import pytest

import paper_1912_10082_gb300 as st


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1912_10082_gb300.build import build

    build()


def est(dim=2, n=255, n_t=256, p=2, **kw):
    return st.request_bytes(st.make_desc(dim, n, n_t, **kw), p)


def documented(dim, n, n_t, p, op="heat", mixed=False, maxit=400, max_basis=2048):
    nh, nnz, tab = 1.0, 1.0, 0.0
    for _ in range(dim):
        nh *= n
        nnz *= 3.0 * n - 2.0
        tab += 12.0 * n * n + 16.0 * n
    m = 200 if op == "convdiff" else 80
    k = min(max_basis + 16, p * (min(maxit, m) + 1))
    csr = nnz * (4.0 + 4 * 8.0 + 4 * 4.0) + 4.0 * (nh + 1)
    blocks = 8.0 * nh * ((3.0 if mixed else 2.0) * k + 12.0 * p)
    if op == "convdiff":
        per_col = 8.0 * nh * 84.0
        blocks += per_col * max(1.0, min(p, 16.0, float(int(4e9 // per_col))))
    return csr + tab + blocks + 8.0 * k * n_t


@pytest.mark.parametrize("dim,n,n_t,p", [(1, 63, 64, 1), (2, 255, 256, 2), (3, 127, 512, 4)])
def test_matches_the_documented_footprint(dim, n, n_t, p):
    assert est(dim, n, n_t, p) == pytest.approx(documented(dim, n, n_t, p), rel=1e-12)
    assert est(dim, n, n_t, p, precision=st.ST_MIXED) == pytest.approx(
        documented(dim, n, n_t, p, mixed=True), rel=1e-12)
    cd = est(dim, n, n_t, p, op=st.ST_CONVDIFF, eps=0.05, beta=(1.0, 0.5, 0.25)[:dim])
    assert cd == pytest.approx(documented(dim, n, n_t, p, op="convdiff"), rel=1e-12)
    assert est(dim, n, n_t, p, maxit=10, max_basis=8) == pytest.approx(
        documented(dim, n, n_t, p, maxit=10, max_basis=8), rel=1e-12)


def test_monotone_in_what_admission_compares():
    base = est()
    assert est(n=127) < base < est(n=383)
    assert est(p=1) < base < est(p=4)
    assert est(n_t=64) < base < est(n_t=1024)
    assert base < est(precision=st.ST_MIXED)
    assert base < est(op=st.ST_CONVDIFF, eps=0.05, beta=(1.0, 0.5, 0.0))
    assert est(max_basis=32) < base
    # the 3D benchmark instance stays well inside one GB300's memory
    assert 1e9 < est(3, 127, 512, 4, precision=st.ST_MIXED) < 50e9


def test_invalid_descriptors_give_zero():
    assert est(p=0) == 0.0
    d = st.make_desc(2, 31, 16)
    d.dim = 0
    assert st.request_bytes(d, 2) == 0.0
    d.dim = 4
    assert st.request_bytes(d, 2) == 0.0
    assert st.lib().st_request_bytes(None, 2) == 0.0
