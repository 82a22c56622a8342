// Allocation-free variant of the FP64 shifted solve W = (A + s M)^{-1} M X.
//
// Some callers must not allocate device memory while they run: code that is
// recording work into a CUDA stream capture of its own, or a real-time or
// embedded loop whose memory is fixed after start-up and where a cudaMalloc
// (which may synchronise the device and can fail at any time) is not allowed.
// st_shift_solve may grow a handle-owned workspace on the call, so it is not
// usable there.  This entry point takes the intermediate tensor of the
// fast-diagonalisation transform from a file-scope device array instead.
#include <cstdio>
#include <mutex>

#include "st_common.cuh"

namespace {

// 4,194,304 doubles = 32 MiB.  With lazy module loading (the default since
// CUDA 12.2) the array is reserved on a device when this file's device code is
// first loaded there, i.e. at the first cudaGetSymbolAddress below (the first
// call of the entry point on that device); from then on it stays reserved
// until the process exits.  Enough for n_h * ncols <= 4,194,304 (e.g. one
// column of the 127^3 grid, or 64 columns of the 255^2 grid).
constexpr size_t kScratchDoubles = size_t(1) << 22;
__device__ __align__(256) double g_fd_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

// Host-side name g_fd_scratch is only a stand-in; the device address is looked
// up once per device with that device current.  The problem's device must be
// current: the cached address belongs to the current device only.
int scratch_address(const st_problem* p, double** out) {
    int dev = 0;
    ST_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return ST_EINVAL;
    if (dev != p->device) {
        st_note_msg("st_shift_solve_noalloc: the problem's device is not the current device");
        return ST_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_fd_scratch);
        if (e != cudaSuccess) {
            st_note_cuda(e, "cudaGetSymbolAddress(g_fd_scratch)", __FILE__, __LINE__);
            return ST_ECUDA;
        }
        g_addr[dev] = static_cast<double*>(ptr);
    }
    *out = g_addr[dev];
    return ST_OK;
}

}  // namespace

extern "C" unsigned long st_shift_solve_noalloc_max(void) { return (unsigned long)kScratchDoubles; }

extern "C" int st_shift_solve_noalloc(st_problem* p, double s, const double* X, int ldx, int ncols, double* W,
                                      int ldw) {
    if (!p || !X || !W || ncols < 1 || ldx < p->n_h || ldw < p->n_h) return ST_EINVAL;
    if (!p->tensor_heat) return ST_ENOTSUP;
    if (!(s > -p->lam_min)) return ST_EINVAL;
    if ((size_t)p->n_h * (size_t)ncols > kScratchDoubles) {
        st_note_msg("st_shift_solve_noalloc: n_h * ncols exceeds the 4194304-double scratch array");
        return ST_EINVAL;
    }
    double* scratch = nullptr;
    ST_TRY(scratch_address(p, &scratch));
    // No launch-variant timing here, whatever the calling thread is doing: the tuner would
    // synchronise and use its own buffers.  The tuned or built-in variants are used as they are.
    StTuneSession* saved = st_tune_set_session(nullptr);
    // every entry of the scratch tensor is written before it is read: nothing to clear
    const int rc = st_fd_apply64(p, FD_MASS_RESOLVENT, s, 1.0, X, ldx, ncols, W, ldw, scratch, p->stream);
    st_tune_set_session(saved);
    return rc;
}
