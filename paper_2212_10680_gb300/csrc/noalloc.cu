// fmlbm_diagnostics_noalloc: the lattice reductions (component masses and the
// residual sums) for callers that must not allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not an option -- a host
// callback or a real-time loop that may not block on the allocator, a process
// whose device memory is fully pre-reserved by another framework's pool, or an
// embedding that forbids allocation after start-up.  Such a caller owns every
// input and output buffer and hands in device pointers; this entry point adds
// no allocation of its own.
//
// The per-block partial sums that fmlbm_diagnostics keeps in a per-handle
// cudaMalloc'd buffer live here in one file-scope __device__ array of fixed
// size (kNoallocScratchDoubles doubles = 512 KiB), which every GPU that loads
// the library keeps until the process exits.  Host code cannot use the array's
// name as a device address, so the first call on each device looks the address
// up with cudaGetSymbolAddress while that device is current and caches it.
#include <cstring>
#include <mutex>

#include "fmlbm.h"
#include "fmlbm_launch.cuh"

using namespace fmlbm;

namespace {

constexpr size_t kNoallocScratchDoubles = size_t(1) << 16;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_partial[kNoallocScratchDoubles];

std::mutex g_setup_mutex;
double* g_partial_ptr[kMaxDevices] = {};

// Once per device, with that device current: the device address of the scratch array.
cudaError_t scratch_address(int device, double** out) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_partial_ptr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partial);
        if (e != cudaSuccess) return e;
        g_partial_ptr[device] = static_cast<double*>(p);
    }
    *out = g_partial_ptr[device];
    return cudaSuccess;
}

template <int ST>
cudaError_t run(const StepArgs& A, int nc, void* rho_prev, int have_prev, double* partial, double* out,
                cudaStream_t s) {
    return launch_reduce<ST>(A, nc, rho_prev, have_prev, partial, out, s);
}

}  // namespace

extern "C" fmlbm_status fmlbm_diagnostics_noalloc(int32_t n_components, int32_t nx, int32_t ny,
                                                  int32_t precision, const void* g_device,
                                                  const float* g0_device, void* rho_prev_device,
                                                  int32_t have_prev, double* out_device, void* cuda_stream) {
    if (n_components < 1 || n_components > FMLBM_MAX_COMPONENTS || nx < 1 || ny < 1 || nx > 65536 ||
        ny > 65536 || !g_device || !rho_prev_device || !out_device)
        return FMLBM_E_INVALID_ARG;
    if (precision < FMLBM_FP64 || precision > FMLBM_BF16DEV) return FMLBM_E_INVALID_ARG;
    if ((precision == FMLBM_FP16DEV || precision == FMLBM_BF16DEV) && !g0_device) return FMLBM_E_INVALID_ARG;
    if ((double)nx * ny * n_components * 9 >= 2147483647.0) return FMLBM_E_INVALID_ARG;
    // the fixed scratch holds one row of n_components + 2 partial sums per 32 x 8 tile
    const size_t need = (size_t)reduce_blocks(nx, ny) * (size_t)(n_components + 2);
    if (need > kNoallocScratchDoubles) return FMLBM_E_INVALID_ARG;

    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices) return FMLBM_E_CUDA;
    double* partial = nullptr;
    if (scratch_address(device, &partial) != cudaSuccess) return FMLBM_E_CUDA;

    StepArgs A;
    std::memset(&A, 0, sizeof(A));
    A.nx = nx;
    A.ny = ny;
    A.gin = g_device;
    A.g0in = g0_device;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e;
    switch (precision) {
        case FMLBM_FP64: e = run<ST_F64>(A, n_components, rho_prev_device, have_prev, partial, out_device, s); break;
        case FMLBM_FP32: e = run<ST_F32>(A, n_components, rho_prev_device, have_prev, partial, out_device, s); break;
        case FMLBM_FP16DEV: e = run<ST_F16DEV>(A, n_components, rho_prev_device, have_prev, partial, out_device, s); break;
        default: e = run<ST_BF16DEV>(A, n_components, rho_prev_device, have_prev, partial, out_device, s); break;
    }
    return e == cudaSuccess ? FMLBM_OK : FMLBM_E_CUDA;
}
