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
// name as a device address, so the first call in each CUDA context (each device,
// and again after that device's context was reset and re-created) looks the address
// up with cudaGetSymbolAddress while the device is current and caches it.
#include <cstring>
#include <mutex>

#include <cudaTypedefs.h>

#include "fmlbm.h"
#include "fmlbm_internal.h"
#include "fmlbm_launch.cuh"

using namespace fmlbm;

namespace {

constexpr size_t kNoallocScratchDoubles = size_t(1) << 16;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_partial[kNoallocScratchDoubles];

std::mutex g_setup_mutex;
double* g_partial_ptr[kMaxDevices] = {};
unsigned long long g_partial_ctx[kMaxDevices] = {};  // the context the cached address belongs to

// The unique id of the current CUDA context (cuCtxGetId, through the runtime's driver entry
// points); 0 when it cannot be had, in which case the address is looked up on every call.
unsigned long long current_context_id() {
    static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(p);
        cudaGetLastError();
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// The device address of the scratch array in the current context, looked up once per
// context (a device whose context was reset and re-created gets a fresh lookup: the
// module, and with it the array, may then sit at another address).
cudaError_t scratch_address(int device, double** out) {
    // the device's primary context exists from here on (cudaSetDevice initialises it and
    // allocates nothing), so the context id below is that of the context used
    cudaError_t e0 = cudaSetDevice(device);
    if (e0 != cudaSuccess) return e0;
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_partial_ptr[device] || ctx == 0 || g_partial_ctx[device] != ctx) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partial);
        if (e != cudaSuccess) return e;
        g_partial_ptr[device] = static_cast<double*>(p);
        g_partial_ctx[device] = ctx;
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
    if (precision < FMLBM_FP64 || precision > FMLBM_BF16DEV_LNF64) return FMLBM_E_INVALID_ARG;
    // the _LNF64 forms store their distributions as the 16-bit forms do
    if (precision == FMLBM_FP16DEV_LNF64) precision = FMLBM_FP16DEV;
    if (precision == FMLBM_BF16DEV_LNF64) precision = FMLBM_BF16DEV;
    if ((precision == FMLBM_FP16DEV || precision == FMLBM_BF16DEV) && !g0_device) return FMLBM_E_INVALID_ARG;
    if ((double)nx * ny > 1073741824.0) return FMLBM_E_INVALID_ARG;
    // the fixed scratch holds one row of n_components + 2 partial sums per 32 x 8 tile
    const size_t need = (size_t)reduce_blocks(nx, ny) * (size_t)(n_components + 2);
    if (need > kNoallocScratchDoubles) return FMLBM_E_INVALID_ARG;

    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices) return FMLBM_E_CUDA;
    // every buffer on the current device and large enough for the lattice
    const size_t nxy = (size_t)nx * ny, nc = (size_t)n_components;
    const bool dev16 = precision == FMLBM_FP16DEV || precision == FMLBM_BF16DEV;
    const size_t real = precision == FMLBM_FP64 ? 8 : 4;
    const size_t g_bytes = dev16 ? nc * 8 * nxy * 2 : nc * 9 * nxy * real;
    if (!fmlbm_internal_usable_device_pointer(g_device, g_bytes, device, dev16 ? 2 : real) ||
        (dev16 && !fmlbm_internal_usable_device_pointer(g0_device, nc * nxy * 4, device, 4)) ||
        !fmlbm_internal_usable_device_pointer(rho_prev_device, nc * nxy * real, device, real) ||
        !fmlbm_internal_usable_device_pointer(out_device, (nc + 2) * 8, device, 8))
        return FMLBM_E_INVALID_ARG;
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
