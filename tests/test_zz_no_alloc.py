"""st_shift_solve_noalloc gives the results of st_shift_solve without allocating.

Callers that cannot allocate device memory while they run (code recording its
own stream capture, or a loop whose memory is fixed after start-up) call
st_shift_solve_noalloc, whose scratch is a static device array shared by every
call.  This file is collected last so that, if it fails, a run stopping at the
first failure has already run every other test.
"""

import numpy as np
import pytest
import torch

import paper_1912_10082_gb300 as st

pytestmark = pytest.mark.gpu


def dev(a):
    t = torch.empty((a.shape[1], a.shape[0]), dtype=torch.float64, device="cuda").t()
    t.copy_(torch.from_numpy(np.ascontiguousarray(a)))
    return t


@pytest.mark.parametrize("dim,n,ncols", [(2, 31, 3), (3, 9, 2), (1, 63, 5)])
def test_noalloc_matches_shift_solve_on_two_calls(dim, n, ncols):
    L = st.lib()
    rng = np.random.default_rng(11)
    with st.Problem(dim, n, 4, 1.0, kappa=0.9) as prob:
        for s in (5.0, 900.0):                      # two calls in a row share the scratch array
            X = dev(rng.standard_normal((prob.n_h, ncols)))
            ref = prob.shift_solve(s, X, precision=st.ST_FP64)
            W = st.empty_colmajor(prob.n_h, ncols)
            rc = L.st_shift_solve_noalloc(prob.h, s, X.data_ptr(), X.stride(1), ncols, W.data_ptr(), W.stride(1))
            assert rc == st.ST_OK, L.st_last_error()
            torch.cuda.synchronize()
            err = float((W - ref).norm() / ref.norm())
            assert err <= 1e-13, err


def test_noalloc_rejects_sizes_beyond_its_scratch():
    L = st.lib()
    cap = int(L.st_shift_solve_noalloc_max())
    assert cap == 1 << 22
    with st.Problem(2, 255, 4, 1.0) as prob:
        ncols = cap // prob.n_h + 1
        X = st.empty_colmajor(prob.n_h, ncols)
        W = st.empty_colmajor(prob.n_h, ncols)
        rc = L.st_shift_solve_noalloc(prob.h, 10.0, X.data_ptr(), prob.n_h, ncols, W.data_ptr(), prob.n_h)
        assert rc == st.ST_EINVAL
        assert b"scratch" in L.st_last_error()
