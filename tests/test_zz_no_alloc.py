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


def noalloc(L, prob, s, X, W):
    return L.st_shift_solve_noalloc(prob.h, s, X.data_ptr(), X.stride(1), X.shape[1], W.data_ptr(), W.stride(1))


@pytest.mark.parametrize("dim,n,ncols", [(2, 31, 3), (3, 9, 2), (1, 63, 5)])
def test_noalloc_matches_shift_solve_on_two_calls(dim, n, ncols):
    L = st.lib()
    rng = np.random.default_rng(11)
    with st.Problem(dim, n, 4, 1.0, kappa=0.9) as prob:
        for s in (5.0, 900.0):                      # two calls in a row share the scratch array
            X = dev(rng.standard_normal((prob.n_h, ncols)))
            ref = prob.shift_solve(s, X, precision=st.ST_FP64)
            W = st.empty_colmajor(prob.n_h, ncols)
            rc = noalloc(L, prob, s, X, W)
            assert rc == st.ST_OK, L.st_last_error()
            torch.cuda.synchronize()
            err = float((W - ref).norm() / ref.norm())
            assert err <= 1e-13, err
            # in place: W and X the same buffer (X is read by the first transform only)
            Xw = X.clone(memory_format=torch.preserve_format)
            rc = noalloc(L, prob, s, Xw, Xw)
            assert rc == st.ST_OK, L.st_last_error()
            torch.cuda.synchronize()
            err = float((Xw - ref).norm() / ref.norm())
            assert err <= 1e-13, err


@pytest.mark.parametrize("dim,n,ncols", [(2, 63, 2), (3, 15, 1)])
def test_noalloc_allocates_nothing_and_records_into_a_stream_capture(dim, n, ncols):
    """After a first call on the device (which loads the device code and reserves the static array), calls change
    no device memory figure and can be recorded into the caller's own stream capture (global capture mode: any
    allocation from any thread during the capture would make it fail); the replayed graph gives the results of
    st_shift_solve."""
    L = st.lib()
    rng = np.random.default_rng(12)
    stream = torch.cuda.Stream()
    with st.Problem(dim, n, 4, 1.0, kappa=1.3, stream=stream) as prob:
        X = dev(rng.standard_normal((prob.n_h, ncols)))
        W = st.empty_colmajor(prob.n_h, ncols)
        s = 7.0
        stream.synchronize()
        assert noalloc(L, prob, s, X, W) == st.ST_OK, L.st_last_error()   # first call: module load
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(3):
            assert noalloc(L, prob, s, X, W) == st.ST_OK, L.st_last_error()
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        g = torch.cuda.CUDAGraph()
        W.zero_()
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=stream, capture_error_mode="global"):
            rc = noalloc(L, prob, s, X, W)
        assert rc == st.ST_OK, L.st_last_error()
        torch.cuda.synchronize()
        assert float(W.abs().max()) == 0.0            # captured, not run
        g.replay()
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            ref = prob.shift_solve(s, X, precision=st.ST_FP64)
        torch.cuda.synchronize()
        err = float((W - ref).norm() / ref.norm())
        assert err <= 1e-13, err
        X2 = dev(rng.standard_normal((prob.n_h, ncols)))
        X.copy_(X2)                                    # the graph reads X at replay
        g.replay()
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            ref2 = prob.shift_solve(s, X2, precision=st.ST_FP64)
        torch.cuda.synchronize()
        assert float((W - ref2).norm() / ref2.norm()) <= 1e-13


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
