// C ABI of libfmlbm (declared in include/fmlbm.h): handle management, mixture
// constants (Appendix C of arXiv:2212.10680), step enqueueing, reductions,
// checkpoints.  All device work runs in the kernels of fmlbm_kernels.cuh.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include <cudaTypedefs.h>

#include "fmlbm.h"
#include "fmlbm_internal.h"
#include "fmlbm_launch.cuh"

using namespace fmlbm;

namespace {

// Asynchronous diagnostics: a ring of result slots, each filled by one reduction (fused
// into the next plain step, or standalone) and read back with its own event.
constexpr int kDiagSlots = 4;
constexpr int kDiagWords = kMaxC + 2 + (int)(sizeof(ErrorLatch) + 7) / 8;

struct DiagSlot {
    int64_t ticket = -1;  // which request owns the slot (-1: none)
    int64_t step = 0;     // the state (steps taken) the request describes
    int have_prev = 0;    // whether a snapshot existed when it was computed
    bool enqueued = false;
};

}  // namespace

struct fmlbm_handle {
    int nc = 0;
    fmlbm_mixture mixture{};
    fmlbm_lattice lattice{};
    MixConst mc{};
    cudaStream_t stream = nullptr;
    int device = 0;
    void* g[2] = {nullptr, nullptr};    // F64/F32: all planes; DEV: 16-bit planes
    float* g0[2] = {nullptr, nullptr};  // DEV: float planes a = 0
    void* F[2] = {nullptr, nullptr};
    int cur = 0;
    void* rho_prev = nullptr;     // storage arithmetic type
    int have_prev = 0;
    void* partial = nullptr;         // kDiagSlots sets of per-strip sums (doubles)
    double* diag_dev = nullptr;      // kDiagSlots x kDiagWords results, then the error latch
    cudaStream_t tail = nullptr;     // final sums and copies of fused requests (non-blocking)
    cudaEvent_t part_ev[kDiagSlots] = {};    // [ticket % kDiagSlots]: partial sums of a fused request written
    cudaEvent_t tail_done[kDiagSlots] = {};  // [ticket % kDiagSlots]: the tail that read them has finished
    double* diag_host = nullptr;     // pinned: kDiagSlots x kDiagWords doubles (results + error latch)
    cudaEvent_t diag_ev[kDiagSlots] = {};
    DiagSlot slot[kDiagSlots];
    int64_t next_ticket = 0;
    int64_t pending = -1;            // ticket asked for the current state, not yet enqueued
    ErrorLatch* err_dev = nullptr;
    ErrorLatch* err_host = nullptr;  // pinned
    int64_t step = 0;
    int tile_y = kTileYSmall;
    int variant = FMLBM_VARIANT_AUTO;
    int sms = 1;                     // multiprocessors of the handle's device
    bool tma_maps = false;           // tensor maps of both buffers were encoded
    bool owns_buffers = true;        // false: g, g0 and F belong to the caller (fmlbm_create_with_buffers)
    long long wait_polls = kMaxPolls;  // bound of a wait for a tile copy (bulk-copy step forms)
    int check_y0 = 0, check_y1 = 0;    // rows the domain check covers (check_y1 = 0: all)
    long long* done = nullptr;         // per-tile step counters of the multi-step kernel
    CUtensorMap tmap[2][2];          // [buffer][0: float planes, 1: 16-bit planes]
    std::string last_error;
};

namespace {

constexpr uint32_t kStateMagic = 0x464d4c42u;  // "FMLB"
constexpr uint32_t kStateVersion = 1;

struct StateHeader {
    uint32_t magic, version;
    int32_t nc, nx, ny, precision;
    int64_t step;
    uint64_t g_bytes, g0_bytes, f_bytes;
};

size_t real_size(int precision) { return precision == FMLBM_FP64 ? 8 : 4; }

// bytes of one distribution buffer (g) and, for the 16-bit forms, of its float g_0 planes
void buffer_bytes(int nc, const fmlbm_lattice& L, size_t* g_bytes, size_t* g0_bytes, size_t* f_bytes) {
    const size_t nxy = (size_t)L.nx * (size_t)L.ny;
    if (L.precision == FMLBM_FP64 || L.precision == FMLBM_FP32) {
        *g_bytes = (size_t)nc * 9 * nxy * real_size(L.precision);
        *g0_bytes = 0;
    } else {
        *g_bytes = (size_t)nc * 8 * nxy * 2;
        *g0_bytes = (size_t)nc * nxy * 4;
    }
    *f_bytes = 2 * nxy * real_size(L.precision);
}

fmlbm_status fail(fmlbm_handle* h, fmlbm_status s, const std::string& msg) {
    if (h) h->last_error = msg;
    return s;
}

fmlbm_status cuda_fail(fmlbm_handle* h, cudaError_t e, const char* where) {
    return fail(h, FMLBM_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define FM_CUDA(h, call)                                      \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call); \
    } while (0)

// Appendix C: a_i = Omega_a R^2 Tc^2 / Pc, b_i = Omega_b R Tc / Pc, alpha_i(T);
// (a alpha)_ij = sqrt((a alpha)_i (a alpha)_j) (1 - k_ij).
bool mixture_constants(const fmlbm_mixture& m, MixConst* mc, std::string* why) {
    const int n = m.n_components;
    if (n < 1 || n > FMLBM_MAX_COMPONENTS) { *why = "n_components must be 1..4"; return false; }
    if (m.eos < 0 || m.eos > 2) { *why = "unknown eos"; return false; }
    if (!(m.R > 0) || !(m.T > 0)) { *why = "R and T must be positive"; return false; }
    double Oa, Ob;
    if (m.eos == FMLBM_EOS_PR) { Oa = 0.457235529; Ob = 0.077796074; }
    else if (m.eos == FMLBM_EOS_SRK) { Oa = 0.4274802; Ob = 0.08664035; }
    else { Oa = 27.0 / 64.0; Ob = 1.0 / 8.0; }
    std::memset(mc, 0, sizeof(*mc));
    mc->nc = n;
    mc->eos = m.eos;
    mc->RT = m.R * m.T;
    double aa[FMLBM_MAX_COMPONENTS];
    for (int i = 0; i < n; ++i) {
        if (!(m.Tc[i] > 0) || !(m.Pc[i] > 0) || !(m.M[i] > 0) || !(m.kappa[i] >= 0)) {
            *why = "Tc, Pc, M must be positive and kappa non-negative";
            return false;
        }
        const double a = Oa * m.R * m.R * m.Tc[i] * m.Tc[i] / m.Pc[i];
        const double b = Ob * m.R * m.Tc[i] / m.Pc[i];
        const double sq = 1.0 - std::sqrt(m.T / m.Tc[i]);
        double alpha = 1.0;
        const double w = m.omega[i];
        if (m.eos == FMLBM_EOS_PR) {
            const double k = w <= 0.49 ? 0.374640 + 1.54226 * w - 0.26992 * w * w
                                       : 0.379642 + 1.48503 * w - 0.164423 * w * w + 0.016666 * w * w * w;
            alpha = (1.0 + k * sq) * (1.0 + k * sq);
        } else if (m.eos == FMLBM_EOS_SRK) {
            const double k = 0.48 + 1.574 * w - 0.176 * w * w;
            alpha = (1.0 + k * sq) * (1.0 + k * sq);
        }
        aa[i] = a * alpha;
        mc->b[i] = b;
        mc->M[i] = m.M[i];
        mc->invM[i] = 1.0 / m.M[i];
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            mc->aij[i * kMaxC + j] = std::sqrt(aa[i] * aa[j]) * (1.0 - m.kij[i * FMLBM_MAX_COMPONENTS + j]);
            mc->kap[i * kMaxC + j] = std::sqrt(m.kappa[i] * m.kappa[j]);
        }
    return true;
}

bool lattice_ok(const fmlbm_lattice& L, int nc, std::string* why) {
    if (L.nx < 1 || L.ny < 1 || L.nx > 65536 || L.ny > 65536) { *why = "nx, ny must be 1..65536"; return false; }
    // node indices within a plane are 32-bit (plane offsets are 64-bit or plane base
    // addresses); the two force planes of a 2^30-node lattice still index below 2^31
    if ((double)L.nx * L.ny > 1073741824.0) { *why = "lattice too large: more than 2^30 nodes"; return false; }
    if (!(L.tau > 0.5)) { *why = "tau must exceed 0.5"; return false; }
    if (L.stencil != FMLBM_STENCIL_ISOTROPIC && L.stencil != FMLBM_STENCIL_CENTRAL) { *why = "unknown stencil"; return false; }
    if (L.precision < FMLBM_FP64 || L.precision > FMLBM_BF16DEV_LNF64) { *why = "unknown precision"; return false; }
    if (L.velocity_force != FMLBM_FORCE_LAGGED && L.velocity_force != FMLBM_FORCE_CURRENT) {
        *why = "unknown velocity_force";
        return false;
    }
    if (L.formulation != FMLBM_WELL_BALANCED && L.formulation != FMLBM_STANDARD) {
        *why = "unknown formulation";
        return false;
    }
    if (L.formulation == FMLBM_STANDARD && L.precision != FMLBM_FP64 && L.precision != FMLBM_FP32) {
        // the 16-bit forms store g_a (a != 0) as deviations from the well-balanced rest
        // state, 0; the standard rest state w_a rho_i would not fit their range
        *why = "the standard formulation needs FP64 or FP32 storage";
        return false;
    }
    return true;
}

StepArgs make_args(const fmlbm_handle* h, int src) {
    StepArgs A;
    std::memset(&A, 0, sizeof(A));
    A.nx = h->lattice.nx;
    A.ny = h->lattice.ny;
    A.stencil = h->lattice.stencil;
    A.lagged = h->lattice.velocity_force == FMLBM_FORCE_LAGGED;
    A.standard = h->lattice.formulation == FMLBM_STANDARD;
    A.gin = h->g[src];
    A.g0in = h->g0[src];
    A.gout = h->g[src ^ 1];
    A.g0out = h->g0[src ^ 1];
    A.Fin = h->F[src];
    A.Fout = h->F[src ^ 1];
    A.err = h->err_dev;
    A.wait_polls = h->wait_polls;
    A.check_y0 = h->check_y0;
    A.check_y1 = h->check_y1;
    MixConst mc = h->mc;
    mc.omega = 1.0 / h->lattice.tau;
    mc.fcoef = 1.0 - 0.5 / h->lattice.tau;
    mc.invRT = 1.0 / mc.RT;
    A.mixd = mc;
    A.mixf = cast_mix<float>(mc);
    return A;
}

bool pair_supported_for(const fmlbm_handle* h) {
    if (h->lattice.formulation != FMLBM_WELL_BALANCED) return false;  // the paired step is well-balanced only
    switch (h->lattice.precision) {
        case FMLBM_FP32: return pair_supported<ST_F32>(h->nc);
        case FMLBM_FP16DEV: return pair_supported<ST_F16DEV>(h->nc);
        case FMLBM_BF16DEV: return pair_supported<ST_BF16DEV>(h->nc);
        default: return false;
    }
}

// The multi-step kernel: float and 16-bit storage with the options of the specialised step.
bool multi_supported_for(const fmlbm_handle* h) {
    const int p = h->lattice.precision;
    return (p == FMLBM_FP32 || p == FMLBM_FP16DEV || p == FMLBM_BF16DEV) && h->mc.eos == 0 &&
           h->lattice.stencil == FMLBM_STENCIL_ISOTROPIC && h->lattice.velocity_force == FMLBM_FORCE_LAGGED &&
           h->lattice.formulation == FMLBM_WELL_BALANCED;
}

bool tma_supported_for(int precision, int nc) {
    switch (precision) {
        case FMLBM_FP32: return tma_supported<ST_F32>(nc);
        case FMLBM_FP16DEV: return tma_supported<ST_F16DEV>(nc);
        case FMLBM_BF16DEV: return tma_supported<ST_BF16DEV>(nc);
        default: return false;
    }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link against libcuda).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// 3-D map (x, y, plane) of one buffer: box = the stage of the TMA step kernel.
bool encode_map(CUtensorMap* map, void* base, CUtensorMapDataType type, size_t esize, int nx, int ny, int planes,
                int box_x, int box_y) {
    auto enc = tensor_map_encoder();
    if (!enc) return false;
    cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)planes};
    cuuint64_t strides[2] = {(cuuint64_t)nx * esize, (cuuint64_t)nx * ny * esize};
    cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, (cuuint32_t)planes};
    cuuint32_t estr[3] = {1, 1, 1};
    return enc(map, type, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor maps for the TMA step, when the layout allows them: 16-byte row strides
// (nx a multiple of 4 for float planes, of 8 for 16-bit planes), planes within the box
// limit, lattices tall and wide enough to have wrap-free tiles.
void setup_tma(fmlbm_handle* h) {
    h->tma_maps = false;
    const int p = h->lattice.precision, nc = h->nc, nx = h->lattice.nx, ny = h->lattice.ny;
    if (!tma_supported_for(p, nc) || nx < kTX + 6 || ny < kTmaTileY + 6) return;
    if (h->lattice.formulation != FMLBM_WELL_BALANCED) return;  // the TMA forms are well-balanced only
    const int H = kTmaTileY + 6;
    bool ok = true;
    for (int b = 0; b < 2 && ok; ++b) {
        if (p == FMLBM_FP32) {
            ok = nx % 4 == 0 && encode_map(&h->tmap[b][0], h->g[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, nx, ny, 9 * nc,
                                           kTX + 8, H);
            h->tmap[b][1] = h->tmap[b][0];
        } else {
            const CUtensorMapDataType t16 =
                p == FMLBM_FP16DEV ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
            ok = nx % 8 == 0 &&
                 encode_map(&h->tmap[b][0], h->g0[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, nx, ny, nc, kTX + 8, H) &&
                 encode_map(&h->tmap[b][1], h->g[b], t16, 2, nx, ny, 8 * nc, kTX + 16, H);
        }
    }
    h->tma_maps = ok;
}

cudaError_t dispatch_step_tma(const fmlbm_handle* h, const StepArgs& A, bool single) {
    const CUtensorMap* maps = h->tmap[h->cur];
    switch (h->lattice.precision) {
        case FMLBM_FP32: return launch_step_tma<ST_F32>(A, h->nc, maps, 1, single, h->stream);
        case FMLBM_FP16DEV: return launch_step_tma<ST_F16DEV>(A, h->nc, maps, 1, single, h->stream);
        case FMLBM_BF16DEV: return launch_step_tma<ST_BF16DEV>(A, h->nc, maps, 1, single, h->stream);
        default: return cudaErrorNotSupported;
    }
}

// AUTO resolves to the plain step: it matched or beat every other form on the workloads
// measured on GB300 (1024^2 binary FP32: 39 us per step against 47 us for the paired step;
// 4096^2 ternary FP32 and BF16 deviations: 1.6x faster than the paired step, which issues
// 40% fewer instructions per node but keeps fewer warps resident); fmlbm_autotune measures
// the lattice at hand instead.  Every form gives the same bits.
int resolved_variant(const fmlbm_handle* h) {
    if (h->variant == FMLBM_VARIANT_AUTO) return FMLBM_VARIANT_PLAIN;
    return h->variant;
}

cudaError_t dispatch_step_pair(const fmlbm_handle* h, const StepArgs& A) {
    switch (h->lattice.precision) {
        case FMLBM_FP32: return launch_step_pair<ST_F32>(A, h->nc, h->stream);
        case FMLBM_FP16DEV: return launch_step_pair<ST_F16DEV>(A, h->nc, h->stream);
        case FMLBM_BF16DEV: return launch_step_pair<ST_BF16DEV>(A, h->nc, h->stream);
        default: return cudaErrorNotSupported;
    }
}

cudaError_t dispatch_step(const fmlbm_handle* h, const StepArgs& A, bool moments) {
    if (!moments) {
        const int v = resolved_variant(h);
        if (v == FMLBM_VARIANT_PAIR) return dispatch_step_pair(h, A);
        if (v == FMLBM_VARIANT_TMA || v == FMLBM_VARIANT_TMA_TILE)
            return dispatch_step_tma(h, A, v == FMLBM_VARIANT_TMA_TILE);
    }
    switch (h->lattice.precision) {
        case FMLBM_FP64: return launch_step<ST_F64>(A, h->nc, moments, h->tile_y, h->stream);
        case FMLBM_FP32: return launch_step<ST_F32>(A, h->nc, moments, h->tile_y, h->stream);
        case FMLBM_FP16DEV: return launch_step<ST_F16DEV>(A, h->nc, moments, h->tile_y, h->stream);
        case FMLBM_FP16DEV_LNF64: return launch_step<ST_F16DEV_X>(A, h->nc, moments, h->tile_y, h->stream);
        case FMLBM_BF16DEV_LNF64: return launch_step<ST_BF16DEV_X>(A, h->nc, moments, h->tile_y, h->stream);
        default: return launch_step<ST_BF16DEV>(A, h->nc, moments, h->tile_y, h->stream);
    }
}
cudaError_t dispatch_init(const fmlbm_handle* h, const StepArgs& A, const double* rho) {
    switch (h->lattice.precision) {
        case FMLBM_FP64: return launch_init<ST_F64>(A, h->nc, rho, h->stream);
        case FMLBM_FP32: return launch_init<ST_F32>(A, h->nc, rho, h->stream);
        case FMLBM_FP16DEV:
        case FMLBM_FP16DEV_LNF64: return launch_init<ST_F16DEV>(A, h->nc, rho, h->stream);
        default: return launch_init<ST_BF16DEV>(A, h->nc, rho, h->stream);
    }
}
cudaError_t dispatch_convert(const fmlbm_handle* h, const StepArgs& A, const double* gi, double* go, bool to) {
    switch (h->lattice.precision) {
        case FMLBM_FP64: return launch_convert<ST_F64>(A, h->nc, gi, go, to, h->stream);
        case FMLBM_FP32: return launch_convert<ST_F32>(A, h->nc, gi, go, to, h->stream);
        case FMLBM_FP16DEV:
        case FMLBM_FP16DEV_LNF64: return launch_convert<ST_F16DEV>(A, h->nc, gi, go, to, h->stream);
        default: return launch_convert<ST_BF16DEV>(A, h->nc, gi, go, to, h->stream);
    }
}
cudaError_t dispatch_reduce(fmlbm_handle* h, const StepArgs& A, void* partial, double* out) {
    switch (h->lattice.precision) {
        case FMLBM_FP64: return launch_reduce<ST_F64>(A, h->nc, h->rho_prev, h->have_prev, partial, out, h->stream);
        case FMLBM_FP32: return launch_reduce<ST_F32>(A, h->nc, h->rho_prev, h->have_prev, partial, out, h->stream);
        case FMLBM_FP16DEV:
        case FMLBM_FP16DEV_LNF64: return launch_reduce<ST_F16DEV>(A, h->nc, h->rho_prev, h->have_prev, partial, out, h->stream);
        default: return launch_reduce<ST_BF16DEV>(A, h->nc, h->rho_prev, h->have_prev, partial, out, h->stream);
    }
}

cudaError_t dispatch_lnrho(fmlbm_handle* h, const StepArgs& A, double* partial, double* out) {
    switch (h->lattice.precision) {
        case FMLBM_FP64: return launch_lnrho<ST_F64>(A, h->nc, partial, out, h->stream);
        case FMLBM_FP32: return launch_lnrho<ST_F32>(A, h->nc, partial, out, h->stream);
        case FMLBM_FP16DEV:
        case FMLBM_FP16DEV_LNF64: return launch_lnrho<ST_F16DEV>(A, h->nc, partial, out, h->stream);
        default: return launch_lnrho<ST_BF16DEV>(A, h->nc, partial, out, h->stream);
    }
}

// Synchronise the stream and turn a latched kernel error into a status.
fmlbm_status sync_and_check(fmlbm_handle* h) {
    FM_CUDA(h, cudaMemcpyAsync(h->err_host, h->err_dev, sizeof(ErrorLatch), cudaMemcpyDeviceToHost, h->stream));
    FM_CUDA(h, cudaStreamSynchronize(h->stream));
    if (h->err_host->flag == 2) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "a bounded wait for a tile copy ran out (tile at x=%d, y=%d)", h->err_host->x,
                      h->err_host->y);
        return fail(h, FMLBM_E_TIMEOUT, buf);
    }
    if (h->err_host->flag) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "node left the EOS domain: component %d at (x=%d, y=%d)", h->err_host->comp,
                      h->err_host->x, h->err_host->y);
        return fail(h, FMLBM_E_NONPHYSICAL, buf);
    }
    return FMLBM_OK;
}

void release(fmlbm_handle* h) {
    for (int k = 0; k < 2 && h->owns_buffers; ++k) {
        if (h->g[k]) cudaFree(h->g[k]);
        if (h->g0[k]) cudaFree(h->g0[k]);
        if (h->F[k]) cudaFree(h->F[k]);
    }
    if (h->rho_prev) cudaFree(h->rho_prev);
    if (h->partial) cudaFree(h->partial);
    if (h->done) cudaFree(h->done);
    if (h->diag_dev) cudaFree(h->diag_dev);
    if (h->diag_host) cudaFreeHost(h->diag_host);
    for (int k = 0; k < kDiagSlots; ++k)
        if (h->diag_ev[k]) cudaEventDestroy(h->diag_ev[k]);
    for (int k = 0; k < kDiagSlots; ++k) {
        if (h->part_ev[k]) cudaEventDestroy(h->part_ev[k]);
        if (h->tail_done[k]) cudaEventDestroy(h->tail_done[k]);
    }
    if (h->tail) cudaStreamDestroy(h->tail);
    if (h->err_host) cudaFreeHost(h->err_host);
}

fmlbm_status reset_state_flags(fmlbm_handle* h) {
    FM_CUDA(h, cudaMemsetAsync(h->err_dev, 0, sizeof(ErrorLatch), h->stream));
    h->have_prev = 0;
    h->step = 0;
    h->cur = 0;
    h->pending = -1;  // a request for the replaced state can no longer be served
    for (int k = 0; k < kDiagSlots; ++k)
        if (!h->slot[k].enqueued) h->slot[k].ticket = -1;
    return FMLBM_OK;
}

// Partial sums of request `ticket`: one set per result slot, so a step that fuses a request
// waits only for the final sum of the request kDiagSlots tickets earlier (with two sets,
// alternating, the 1024^2 binary's end-to-end loop stalled for the previous request's
// final sum, which gets SMs only as the running step drains).
void* partial_set(const fmlbm_handle* h, int64_t ticket) {
    return static_cast<char*>(h->partial) +
           (size_t)(ticket % kDiagSlots) * reduce_blocks(h->lattice.nx, h->lattice.ny) * (kMaxC + 2) * sizeof(double);
}
double* result_slot(const fmlbm_handle* h, int64_t ticket) { return h->diag_dev + (ticket % kDiagSlots) * kDiagWords; }

// Final sum of request `ticket` (unless already done; its partial sums are enqueued ahead
// on stream s), copy of the results and of the error latch into its host slot, event.
fmlbm_status enqueue_diag_tail(fmlbm_handle* h, int64_t ticket, cudaStream_t s, bool final_sum, bool capturing) {
    DiagSlot& sl = h->slot[ticket % kDiagSlots];
    double* host = h->diag_host + (size_t)(ticket % kDiagSlots) * kDiagWords;
    // the final sum writes the sums and, after them, the error latch into the result slot
    // (the standalone reduction did the same), so one copy brings both to the host
    if (final_sum)
        FM_CUDA(h, launch_reduce_final(h->nc, partial_set(h, ticket), h->lattice.nx, h->lattice.ny,
                                       result_slot(h, ticket), s, h->err_dev));
    FM_CUDA(h, cudaMemcpyAsync(host, result_slot(h, ticket), kDiagWords * sizeof(double), cudaMemcpyDeviceToHost, s));
    // inside a stream capture the record becomes a node of the graph (an external event),
    // so fmlbm_diagnostics_wait can wait for it after the graph is launched
    if (capturing)
        FM_CUDA(h, cudaEventRecordWithFlags(h->diag_ev[ticket % kDiagSlots], s, cudaEventRecordExternal));
    else
        FM_CUDA(h, cudaEventRecord(h->diag_ev[ticket % kDiagSlots], s));
    sl.have_prev = h->have_prev;
    sl.enqueued = true;
    h->have_prev = 1;
    h->pending = -1;
    return FMLBM_OK;
}

// The pending request served by a standalone reduction of the current state (all on the
// handle's stream, after any tail still reading the same set of partial sums).
fmlbm_status enqueue_pending_standalone(fmlbm_handle* h) {
    if (h->pending < 0) return FMLBM_OK;
    const int64_t t = h->pending;
    StepArgs A = make_args(h, h->cur);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    FM_CUDA(h, cudaStreamIsCapturing(h->stream, &cap));
    const bool capturing = cap != cudaStreamCaptureStatusNone;
    if (!capturing) FM_CUDA(h, cudaStreamWaitEvent(h->stream, h->tail_done[t % kDiagSlots], 0));
    FM_CUDA(h, dispatch_reduce(h, A, partial_set(h, t), result_slot(h, t)));
    return enqueue_diag_tail(h, t, h->stream, false, capturing);
}

// Caller-provided distribution and force buffers (fmlbm_create_with_buffers).
struct ExternalBuffers {
    void* g[2];
    float* g0[2];
    void* F[2];
};

// cuMemGetAddressRange through the runtime's driver entry point: the base and size of the
// allocation that contains a device address (null if the driver does not provide it).
PFN_cuMemGetAddressRange_v3020 address_range_fn() {
    static PFN_cuMemGetAddressRange_v3020 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &p, 3020, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuMemGetAddressRange_v3020>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// Byte ranges [p, p + bytes) that must not overlap (null entries are skipped).
bool disjoint(const void* const* p, const size_t* bytes, int n) {
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            if (!p[i] || !p[j] || !bytes[i] || !bytes[j]) continue;
            const uintptr_t a0 = reinterpret_cast<uintptr_t>(p[i]), b0 = reinterpret_cast<uintptr_t>(p[j]);
            if (a0 < b0 + bytes[j] && b0 < a0 + bytes[i]) return false;
        }
    return true;
}

fmlbm_status create_handle(const fmlbm_mixture* mixture, const fmlbm_lattice* lattice, void* cuda_stream,
                           const ExternalBuffers* ext, fmlbm_handle** out) {
    if (!mixture || !lattice || !out) return FMLBM_E_INVALID_ARG;
    *out = nullptr;
    fmlbm_handle* h = new (std::nothrow) fmlbm_handle();
    if (!h) return FMLBM_E_OOM;
    std::string why;
    if (!mixture_constants(*mixture, &h->mc, &why) || !lattice_ok(*lattice, mixture->n_components, &why)) {
        delete h;
        return FMLBM_E_INVALID_ARG;
    }
    h->nc = mixture->n_components;
    h->mixture = *mixture;
    h->lattice = *lattice;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    h->tile_y = kTileYSmall;
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        delete h;
        return FMLBM_E_CUDA;
    }
    size_t gb, g0b, fb;
    buffer_bytes(h->nc, h->lattice, &gb, &g0b, &fb);
    const size_t nxy = (size_t)lattice->nx * lattice->ny;
    bool ok = true;
    if (ext) {
        h->owns_buffers = false;
        for (int k = 0; k < 2; ++k) {
            const bool g0_ok = g0b ? fmlbm_internal_usable_device_pointer(ext->g0[k], g0b, h->device)
                                   : ext->g0[k] == nullptr;
            if (!fmlbm_internal_usable_device_pointer(ext->g[k], gb, h->device) || !g0_ok ||
                !fmlbm_internal_usable_device_pointer(ext->F[k], fb, h->device)) {
                delete h;
                return FMLBM_E_INVALID_ARG;
            }
            h->g[k] = ext->g[k];
            h->g0[k] = ext->g0[k];
            h->F[k] = ext->F[k];
        }
        // the step reads one buffer of each pair while it writes the other
        const void* ptrs[6] = {ext->g[0], ext->g[1], ext->g0[0], ext->g0[1], ext->F[0], ext->F[1]};
        const size_t sizes[6] = {gb, gb, g0b, g0b, fb, fb};
        if (!disjoint(ptrs, sizes, 6)) {
            delete h;
            return FMLBM_E_INVALID_ARG;
        }
    }
    for (int k = 0; k < 2 && ok && !ext; ++k) {
        ok = ok && cudaMalloc(&h->g[k], gb) == cudaSuccess;
        if (g0b) ok = ok && cudaMalloc((void**)&h->g0[k], g0b) == cudaSuccess;
        ok = ok && cudaMalloc(&h->F[k], fb) == cudaSuccess;
    }
    ok = ok && cudaMalloc(&h->rho_prev, (size_t)h->nc * nxy * real_size(lattice->precision)) == cudaSuccess;
    ok = ok && cudaMalloc(&h->partial, kDiagSlots * (size_t)reduce_blocks(lattice->nx, lattice->ny) * (kMaxC + 2) *
                                           sizeof(double)) == cudaSuccess;
    ok = ok && cudaMalloc((void**)&h->diag_dev, (kDiagSlots * kDiagWords + 2) * sizeof(double)) == cudaSuccess;
    if (ok) h->err_dev = reinterpret_cast<ErrorLatch*>(h->diag_dev + kDiagSlots * kDiagWords);
    // the diagnostics stream at the highest priority: its small final sums are dispatched as
    // soon as the running step frees a block slot, instead of after the step's last block
    int prio_least = 0, prio_greatest = 0;
    ok = ok && cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest) == cudaSuccess;
    ok = ok && cudaStreamCreateWithPriority(&h->tail, cudaStreamNonBlocking, prio_greatest) == cudaSuccess;
    for (int k = 0; k < kDiagSlots; ++k) {
        ok = ok && cudaEventCreateWithFlags(&h->part_ev[k], cudaEventDisableTiming) == cudaSuccess;
        ok = ok && cudaEventCreateWithFlags(&h->tail_done[k], cudaEventDisableTiming) == cudaSuccess;
    }
    ok = ok && cudaMallocHost((void**)&h->diag_host, (size_t)kDiagSlots * kDiagWords * sizeof(double)) == cudaSuccess;
    for (int k = 0; k < kDiagSlots; ++k)
        ok = ok && cudaEventCreateWithFlags(&h->diag_ev[k], cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaMallocHost((void**)&h->err_host, sizeof(ErrorLatch)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        release(h);
        delete h;
        return FMLBM_E_OOM;
    }
    if (cudaMemsetAsync(h->err_dev, 0, sizeof(ErrorLatch), h->stream) != cudaSuccess) {
        release(h);
        delete h;
        return FMLBM_E_CUDA;
    }
    cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
    setup_tma(h);
    *out = h;
    return FMLBM_OK;
}

}  // namespace

// A device (or managed) allocation of this process on `device`, aligned to `align` bytes (a
// power of two), with at
// least `bytes` from p to the end of the allocation that contains it (a buffer carved out
// of a larger pool allocation is checked against the pool allocation).  Memory of another
// GPU is refused: a kernel would reach it over NVLink with peer access, or fault without.
bool fmlbm_internal_usable_device_pointer(const void* p, size_t bytes, int device, size_t align) {
    if (!p || (reinterpret_cast<uintptr_t>(p) & (align - 1)) != 0) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return false;
    if (a.type == cudaMemoryTypeDevice && a.device != device) return false;
    if (auto range = address_range_fn()) {
        CUdeviceptr base = 0;
        size_t size = 0;
        const CUdeviceptr d = reinterpret_cast<CUdeviceptr>(p);
        if (range(&base, &size, d) != CUDA_SUCCESS) return false;
        if (d + bytes > base + size) return false;
    }
    return true;
}

void fmlbm_internal_set_check_rows(fmlbm_handle* h, int y0, int y1) {
    h->check_y0 = y0;
    h->check_y1 = y1;
}

bool fmlbm_internal_mixture_constants(const fmlbm_mixture& m, MixConst* mc, std::string* why) {
    return mixture_constants(m, mc, why);
}
bool fmlbm_internal_lattice_ok(const fmlbm_lattice& L, int nc, std::string* why) { return lattice_ok(L, nc, why); }

extern "C" {

const char* fmlbm_version(void) { return "fmlbm 0.1 sm_103a"; }

const char* fmlbm_status_str(fmlbm_status s) {
    switch (s) {
        case FMLBM_OK: return "FMLBM_OK";
        case FMLBM_E_INVALID_ARG: return "FMLBM_E_INVALID_ARG";
        case FMLBM_E_OOM: return "FMLBM_E_OOM";
        case FMLBM_E_CUDA: return "FMLBM_E_CUDA";
        case FMLBM_E_NONPHYSICAL: return "FMLBM_E_NONPHYSICAL";
        case FMLBM_E_TIMEOUT: return "FMLBM_E_TIMEOUT";
        case FMLBM_E_BUSY: return "FMLBM_E_BUSY";
        case FMLBM_E_NOT_CONVERGED: return "FMLBM_E_NOT_CONVERGED";
        case FMLBM_E_UNSUPPORTED: return "FMLBM_E_UNSUPPORTED";
    }
    return "unknown fmlbm_status";
}

const char* fmlbm_last_error(const fmlbm_handle* h) { return h ? h->last_error.c_str() : ""; }

fmlbm_status fmlbm_lattice_bytes(int32_t n_components, const fmlbm_lattice* lattice, size_t* bytes) {
    if (!lattice || !bytes || n_components < 1 || n_components > FMLBM_MAX_COMPONENTS) return FMLBM_E_INVALID_ARG;
    size_t gb, g0b, fb;
    buffer_bytes(n_components, *lattice, &gb, &g0b, &fb);
    const size_t nxy = (size_t)lattice->nx * lattice->ny;
    *bytes = 2 * (gb + g0b + fb) + (size_t)n_components * nxy * real_size(lattice->precision) +
             kDiagSlots * (size_t)reduce_blocks(lattice->nx, lattice->ny) * (FMLBM_MAX_COMPONENTS + 2) * 8 + 512;
    return FMLBM_OK;
}


fmlbm_status fmlbm_create(const fmlbm_mixture* mixture, const fmlbm_lattice* lattice, void* cuda_stream,
                          fmlbm_handle** out) {
    return create_handle(mixture, lattice, cuda_stream, nullptr, out);
}

fmlbm_status fmlbm_create_with_buffers(const fmlbm_mixture* mixture, const fmlbm_lattice* lattice, void* cuda_stream,
                                       void* const g[2], float* const g0[2], void* const force[2],
                                       fmlbm_handle** out) {
    if (!g || !force) return FMLBM_E_INVALID_ARG;
    ExternalBuffers ext;
    for (int k = 0; k < 2; ++k) {
        ext.g[k] = g[k];
        ext.g0[k] = g0 ? g0[k] : nullptr;
        ext.F[k] = force[k];
    }
    return create_handle(mixture, lattice, cuda_stream, &ext, out);
}

fmlbm_status fmlbm_buffer_sizes(int32_t n_components, const fmlbm_lattice* lattice, size_t* g_bytes,
                                size_t* g0_bytes, size_t* force_bytes) {
    if (!lattice || !g_bytes || !g0_bytes || !force_bytes || n_components < 1 ||
        n_components > FMLBM_MAX_COMPONENTS)
        return FMLBM_E_INVALID_ARG;
    std::string why;
    if (!lattice_ok(*lattice, n_components, &why)) return FMLBM_E_INVALID_ARG;
    buffer_bytes(n_components, *lattice, g_bytes, g0_bytes, force_bytes);
    return FMLBM_OK;
}

void fmlbm_destroy(fmlbm_handle* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    if (h->tail) cudaStreamSynchronize(h->tail);
    release(h);
    delete h;
}

fmlbm_status fmlbm_init_device(fmlbm_handle* h, const double* rho_device) {
    if (!h || !rho_device) return fail(h, FMLBM_E_INVALID_ARG, "null argument");
    fmlbm_status s = reset_state_flags(h);
    if (s != FMLBM_OK) return s;
    StepArgs A = make_args(h, 1);  // writes into buffer 0
    FM_CUDA(h, dispatch_init(h, A, rho_device));
    h->cur = 0;
    return FMLBM_OK;
}

fmlbm_status fmlbm_init(fmlbm_handle* h, const double* rho_host) {
    if (!h || !rho_host) return fail(h, FMLBM_E_INVALID_ARG, "null argument");
    const size_t bytes = (size_t)h->nc * h->lattice.nx * h->lattice.ny * sizeof(double);
    // Page-locked host memory that this context has mapped: the initialisation kernel reads the
    // densities in place (over the device's link to host memory; no device copy, no allocation),
    // and the call waits for it so that the buffer is free again on return.
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, rho_host) == cudaSuccess && at.type == cudaMemoryTypeHost &&
        at.devicePointer != nullptr) {
        fmlbm_status s = fmlbm_init_device(h, static_cast<const double*>(at.devicePointer));
        if (s != FMLBM_OK) return s;
        FM_CUDA(h, cudaStreamSynchronize(h->stream));
        return FMLBM_OK;
    }
    cudaGetLastError();  // an unregistered pointer leaves no error behind
    double* d = nullptr;
    FM_CUDA(h, cudaMallocAsync((void**)&d, bytes, h->stream));
    cudaError_t e = cudaMemcpyAsync(d, rho_host, bytes, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) {
        cudaFreeAsync(d, h->stream);
        return cuda_fail(h, e, "cudaMemcpyAsync(rho)");
    }
    fmlbm_status s = fmlbm_init_device(h, d);
    cudaFreeAsync(d, h->stream);
    return s;
}

fmlbm_status fmlbm_step(fmlbm_handle* h, int64_t nsteps) {
    if (!h || nsteps < 0) return fail(h, FMLBM_E_INVALID_ARG, "bad argument");
    // During a stream capture nothing crosses to the diagnostics stream (a captured stream
    // may not wait on work outside the capture): a request is then served entirely on the
    // captured stream.
    bool capturing = false;
    if (nsteps > 0 && h->pending >= 0) {
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        FM_CUDA(h, cudaStreamIsCapturing(h->stream, &cap));
        capturing = cap != cudaStreamCaptureStatusNone;
    }
    for (int64_t k = 0; k < nsteps; ++k) {
        if (nsteps - k >= 2 && h->pending < 0 && resolved_variant(h) == FMLBM_VARIANT_MULTI) {
            // the remaining steps in one launch (at most 2^30 per launch)
            if (!h->done)
                FM_CUDA(h, cudaMalloc(&h->done, (size_t)multi_tiles(h->lattice.nx, h->lattice.ny) * sizeof(long long)));
            const int64_t left = nsteps - k;
            const int n = left > (int64_t(1) << 30) ? (1 << 30) : (int)left;
            const StepArgs A0 = make_args(h, h->cur), A1 = make_args(h, h->cur ^ 1);
            cudaError_t e;
            switch (h->lattice.precision) {
                case FMLBM_FP32: e = launch_steps_multi<ST_F32>(A0, A1, h->nc, n, h->done, h->stream); break;
                case FMLBM_FP16DEV: e = launch_steps_multi<ST_F16DEV>(A0, A1, h->nc, n, h->done, h->stream); break;
                default: e = launch_steps_multi<ST_BF16DEV>(A0, A1, h->nc, n, h->done, h->stream); break;
            }
            FM_CUDA(h, e);
            h->cur ^= n & 1;
            h->step += n;
            k += n - 1;
            continue;
        }
        StepArgs A = make_args(h, h->cur);
        const int64_t fused = h->pending;
        if (fused >= 0) {  // this step also reduces the state it reads
            A.diag_partial = partial_set(h, fused);
            A.rho_prev = h->rho_prev;
            A.have_prev = h->have_prev;
            // the tail of request fused - kDiagSlots may still read this set of partial sums
            if (!capturing) FM_CUDA(h, cudaStreamWaitEvent(h->stream, h->tail_done[fused % kDiagSlots], 0));
        }
        FM_CUDA(h, dispatch_step(h, A, false));
        if (fused >= 0) {
            // final sum and copies on the diagnostics stream, so the next step need not wait
            cudaStream_t ts = h->stream;
            if (!capturing) {
                FM_CUDA(h, cudaEventRecord(h->part_ev[fused % kDiagSlots], h->stream));
                FM_CUDA(h, cudaStreamWaitEvent(h->tail, h->part_ev[fused % kDiagSlots], 0));
                ts = h->tail;
            }
            fmlbm_status s = enqueue_diag_tail(h, fused, ts, true, capturing);
            if (s != FMLBM_OK) return s;
            if (!capturing) FM_CUDA(h, cudaEventRecord(h->tail_done[fused % kDiagSlots], ts));
        }
        h->cur ^= 1;
        ++h->step;
    }
    return FMLBM_OK;
}

fmlbm_status fmlbm_step(fmlbm_handle* h, int64_t nsteps);

fmlbm_status fmlbm_set_tile_height(fmlbm_handle* h, int32_t tile_y) {
    if (!h || (tile_y != kTileYSmall && tile_y != kTileYLarge && tile_y != kTileYHuge))
        return fail(h, FMLBM_E_INVALID_ARG, "tile height must be 8, 16 or 32");
    h->tile_y = tile_y;
    return FMLBM_OK;
}

fmlbm_status fmlbm_set_step_variant(fmlbm_handle* h, int32_t variant) {
    if (!h || variant < FMLBM_VARIANT_AUTO || variant > FMLBM_VARIANT_MULTI)
        return fail(h, FMLBM_E_INVALID_ARG, "unknown step variant");
    if ((variant == FMLBM_VARIANT_TMA || variant == FMLBM_VARIANT_TMA_TILE) && !h->tma_maps)
        return fail(h, FMLBM_E_UNSUPPORTED, "no TMA step for this precision, component count or lattice shape");
    if (variant == FMLBM_VARIANT_PAIR && !pair_supported_for(h))
        return fail(h, FMLBM_E_UNSUPPORTED, "no paired step for this precision or formulation");
    if (variant == FMLBM_VARIANT_MULTI && !multi_supported_for(h))
        return fail(h, FMLBM_E_UNSUPPORTED, "no multi-step kernel for this precision, EOS or options");
    h->variant = variant;
    return FMLBM_OK;
}

fmlbm_status fmlbm_autotune(fmlbm_handle* h, int32_t steps_per_trial, int32_t* variant, int32_t* tile_y,
                            double* ms_per_step) {
    if (!h || steps_per_trial < 1) return fail(h, FMLBM_E_INVALID_ARG, "bad argument");
    struct Cand { int variant, tile_y; };
    Cand cands[7];
    int nc = 0;
    if (steps_per_trial >= 2 && multi_supported_for(h)) cands[nc++] = Cand{FMLBM_VARIANT_MULTI, kTileYSmall};
    if (pair_supported_for(h)) cands[nc++] = Cand{FMLBM_VARIANT_PAIR, kTileYSmall};
    for (int ty : {kTileYSmall, kTileYLarge, kTileYHuge})
        if (ty <= 16 || h->lattice.ny >= 64) cands[nc++] = Cand{FMLBM_VARIANT_PLAIN, ty};
    if (h->tma_maps) {
        cands[nc++] = Cand{FMLBM_VARIANT_TMA, h->tile_y};
        cands[nc++] = Cand{FMLBM_VARIANT_TMA_TILE, h->tile_y};
    }
    cudaEvent_t e0, e1;
    FM_CUDA(h, cudaEventCreate(&e0));
    FM_CUDA(h, cudaEventCreate(&e1));
    float best = 1e30f;
    Cand pick = cands[0];
    for (int k = 0; k < nc; ++k) {
        h->variant = cands[k].variant;
        h->tile_y = cands[k].tile_y;
        // every trial step is a real step: the variants give bit-identical results
        fmlbm_status st = fmlbm_step(h, 1);
        if (st != FMLBM_OK) return st;
        FM_CUDA(h, cudaEventRecord(e0, h->stream));
        st = fmlbm_step(h, steps_per_trial);
        if (st != FMLBM_OK) return st;
        FM_CUDA(h, cudaEventRecord(e1, h->stream));
        FM_CUDA(h, cudaEventSynchronize(e1));
        float ms = 0.f;
        FM_CUDA(h, cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) {
            best = ms;
            pick = cands[k];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->variant = pick.variant;
    h->tile_y = pick.tile_y;
    if (variant) *variant = pick.variant;
    if (tile_y) *tile_y = pick.tile_y;
    if (ms_per_step) *ms_per_step = best / steps_per_trial;
    return sync_and_check(h);
}

fmlbm_status fmlbm_set_wait_limit(fmlbm_handle* h, int64_t polls) {
    if (!h || polls < 0) return fail(h, FMLBM_E_INVALID_ARG, "the wait limit must be >= 0");
    h->wait_polls = (long long)polls;
    return FMLBM_OK;
}

fmlbm_status fmlbm_get_step_variant(fmlbm_handle* h, int32_t* variant) {
    if (!h || !variant) return FMLBM_E_INVALID_ARG;
    *variant = resolved_variant(h);
    return FMLBM_OK;
}

fmlbm_status fmlbm_synchronize(fmlbm_handle* h) {
    if (!h) return FMLBM_E_INVALID_ARG;
    FM_CUDA(h, cudaStreamSynchronize(h->tail));
    return sync_and_check(h);
}

fmlbm_status fmlbm_moments(fmlbm_handle* h, double* rho, double* u, double* lnf) {
    if (!h) return FMLBM_E_INVALID_ARG;
    const size_t nxy = (size_t)h->lattice.nx * h->lattice.ny;
    const size_t fb = (size_t)h->nc * nxy * sizeof(double);
    double* d = nullptr;
    FM_CUDA(h, cudaMallocAsync((void**)&d, 2 * fb + 2 * nxy * sizeof(double), h->stream));
    StepArgs A = make_args(h, h->cur);
    A.rho_out = d;
    A.lnf_out = d + (size_t)h->nc * nxy;
    A.u_out = d + 2 * (size_t)h->nc * nxy;
    A.gout = nullptr;
    A.g0out = nullptr;
    A.Fout = nullptr;
    cudaError_t e = dispatch_step(h, A, true);
    if (e == cudaSuccess && rho) e = cudaMemcpyAsync(rho, A.rho_out, fb, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && lnf) e = cudaMemcpyAsync(lnf, A.lnf_out, fb, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && u) e = cudaMemcpyAsync(u, A.u_out, 2 * nxy * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    cudaFreeAsync(d, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "moments");
    return sync_and_check(h);
}

fmlbm_status fmlbm_phase_measure(fmlbm_handle* h, double* lambda) {
    if (!h || !lambda) return fail(h, FMLBM_E_INVALID_ARG, "null argument");
    const size_t nb = (size_t)reduce_blocks(h->lattice.nx, h->lattice.ny);
    double* d = nullptr;
    FM_CUDA(h, cudaMallocAsync((void**)&d, (nb + 1) * h->nc * sizeof(double), h->stream));
    double* out = d + nb * h->nc;
    const StepArgs A = make_args(h, h->cur);
    double sums[kMaxC] = {};
    cudaError_t e = dispatch_lnrho(h, A, d, out);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sums, out, h->nc * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    cudaFreeAsync(d, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "phase measure");
    const fmlbm_status st = sync_and_check(h);
    if (st != FMLBM_OK) return st;
    const double n = (double)h->lattice.nx * (double)h->lattice.ny;
    for (int i = 0; i < h->nc; ++i) lambda[i] = sums[i] / n;
    return FMLBM_OK;
}

fmlbm_status fmlbm_get_distributions(fmlbm_handle* h, double* g, double* force) {
    if (!h) return FMLBM_E_INVALID_ARG;
    const size_t nxy = (size_t)h->lattice.nx * h->lattice.ny;
    cudaError_t e = cudaSuccess;
    if (g) {
        const size_t gbytes = (size_t)h->nc * 9 * nxy * sizeof(double);
        double* d = nullptr;
        FM_CUDA(h, cudaMallocAsync((void**)&d, gbytes, h->stream));
        StepArgs A = make_args(h, h->cur);
        e = dispatch_convert(h, A, nullptr, d, false);
        if (e == cudaSuccess) e = cudaMemcpyAsync(g, d, gbytes, cudaMemcpyDeviceToHost, h->stream);
        cudaFreeAsync(d, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "get_distributions");
    }
    if (force) {
        if (h->lattice.precision == FMLBM_FP64) {
            FM_CUDA(h, cudaMemcpyAsync(force, h->F[h->cur], 2 * nxy * 8, cudaMemcpyDeviceToHost, h->stream));
            FM_CUDA(h, cudaStreamSynchronize(h->stream));
        } else {
            float* tmp = new (std::nothrow) float[2 * nxy];
            if (!tmp) return FMLBM_E_OOM;
            e = cudaMemcpyAsync(tmp, h->F[h->cur], 2 * nxy * 4, cudaMemcpyDeviceToHost, h->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
            if (e == cudaSuccess)
                for (size_t k = 0; k < 2 * nxy; ++k) force[k] = tmp[k];
            delete[] tmp;
            if (e != cudaSuccess) return cuda_fail(h, e, "get force");
        }
    }
    return sync_and_check(h);
}

fmlbm_status fmlbm_set_distributions(fmlbm_handle* h, const double* g, const double* force) {
    if (!h || !g) return fail(h, FMLBM_E_INVALID_ARG, "null argument");
    fmlbm_status s = reset_state_flags(h);
    if (s != FMLBM_OK) return s;
    const size_t nxy = (size_t)h->lattice.nx * h->lattice.ny;
    const size_t gbytes = (size_t)h->nc * 9 * nxy * sizeof(double);
    double* d = nullptr;
    FM_CUDA(h, cudaMallocAsync((void**)&d, gbytes, h->stream));
    cudaError_t e = cudaMemcpyAsync(d, g, gbytes, cudaMemcpyHostToDevice, h->stream);
    StepArgs A = make_args(h, 1);  // writes buffer 0
    if (e == cudaSuccess) e = dispatch_convert(h, A, d, nullptr, true);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFreeAsync(d, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "set_distributions");
    const size_t rs = real_size(h->lattice.precision);
    if (!force) {
        FM_CUDA(h, cudaMemsetAsync(h->F[0], 0, 2 * nxy * rs, h->stream));
    } else if (rs == 8) {
        FM_CUDA(h, cudaMemcpyAsync(h->F[0], force, 2 * nxy * 8, cudaMemcpyHostToDevice, h->stream));
    } else {
        float* tmp = new (std::nothrow) float[2 * nxy];
        if (!tmp) return FMLBM_E_OOM;
        for (size_t k = 0; k < 2 * nxy; ++k) tmp[k] = (float)force[k];
        e = cudaMemcpyAsync(h->F[0], tmp, 2 * nxy * 4, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        delete[] tmp;
        if (e != cudaSuccess) return cuda_fail(h, e, "set force");
    }
    return sync_and_check(h);
}

fmlbm_status fmlbm_diagnostics_async(fmlbm_handle* h, int64_t* ticket) {
    if (!h || !ticket) return fail(h, FMLBM_E_INVALID_ARG, "null argument");
    if (h->pending < 0) {
        const int64_t t = h->next_ticket++;
        DiagSlot& sl = h->slot[t % kDiagSlots];
        sl.ticket = t;
        sl.step = h->step;
        sl.enqueued = false;
        h->pending = t;
    }
    *ticket = h->pending;  // repeated requests for one state share a ticket
    return FMLBM_OK;
}

fmlbm_status fmlbm_diagnostics_wait(fmlbm_handle* h, int64_t ticket, double* mass, double* residual, int64_t* step) {
    if (!h || ticket < 0) return fail(h, FMLBM_E_INVALID_ARG, "bad argument");
    DiagSlot& sl = h->slot[ticket % kDiagSlots];
    if (sl.ticket != ticket) return fail(h, FMLBM_E_INVALID_ARG, "unknown or expired diagnostics ticket");
    if (!sl.enqueued) {
        fmlbm_status s = enqueue_pending_standalone(h);  // no step has served it yet
        if (s != FMLBM_OK) return s;
    }
    FM_CUDA(h, cudaEventSynchronize(h->diag_ev[ticket % kDiagSlots]));
    const double* d = h->diag_host + (size_t)(ticket % kDiagSlots) * kDiagWords;
    ErrorLatch latch;
    std::memcpy(&latch, d + kMaxC + 2, sizeof latch);
    if (mass)
        for (int i = 0; i < h->nc; ++i) mass[i] = d[i];
    if (residual) *residual = sl.have_prev ? std::sqrt(d[h->nc]) / std::sqrt(d[h->nc + 1]) : INFINITY;
    if (step) *step = sl.step;
    if (latch.flag == 2) return fail(h, FMLBM_E_TIMEOUT, "a bounded wait for a tile copy ran out");
    if (latch.flag) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "node left the EOS domain: component %d at (x=%d, y=%d)", latch.comp, latch.x,
                      latch.y);
        return fail(h, FMLBM_E_NONPHYSICAL, buf);
    }
    return FMLBM_OK;
}

fmlbm_status fmlbm_diagnostics(fmlbm_handle* h, double* mass, double* residual, int64_t* step) {
    if (!h) return FMLBM_E_INVALID_ARG;
    int64_t t = -1;
    fmlbm_status s = fmlbm_diagnostics_async(h, &t);
    if (s != FMLBM_OK) return s;
    return fmlbm_diagnostics_wait(h, t, mass, residual, step);
}

fmlbm_status fmlbm_step_diagnostics(fmlbm_handle* h, int64_t nsteps, double* mass, double* residual) {
    if (!h || nsteps < 0 || (nsteps > 0 && (!mass || !residual))) return fail(h, FMLBM_E_INVALID_ARG, "bad argument");
    // the per-step loop of fmlbm_diagnostics_async / fmlbm_step / fmlbm_diagnostics_wait, with
    // each result read three steps behind (the four kept results), so that the device always has
    // steps queued while the host reads
    constexpr int64_t kBehind = kDiagSlots - 1;
    int64_t tickets[kDiagSlots];
    fmlbm_status first_error = FMLBM_OK;
    auto read = [&](int64_t k) {
        const fmlbm_status s = fmlbm_diagnostics_wait(h, tickets[k % kDiagSlots], mass + k * h->nc, residual + k,
                                                      nullptr);
        if (s != FMLBM_OK && first_error == FMLBM_OK) first_error = s;
        return s;
    };
    for (int64_t k = 0; k < nsteps; ++k) {
        fmlbm_status s = fmlbm_diagnostics_async(h, &tickets[k % kDiagSlots]);
        if (s == FMLBM_OK) s = fmlbm_step(h, 1);
        if (s != FMLBM_OK) return s;
        if (k >= kBehind && read(k - kBehind) != FMLBM_OK) return first_error;
    }
    for (int64_t k = nsteps > kBehind ? nsteps - kBehind : 0; k < nsteps; ++k)
        if (read(k) != FMLBM_OK) return first_error;
    return FMLBM_OK;
}

fmlbm_status fmlbm_error_node(fmlbm_handle* h, int32_t* comp, int32_t* x, int32_t* y) {
    if (!h) return FMLBM_E_INVALID_ARG;
    FM_CUDA(h, cudaMemcpyAsync(h->err_host, h->err_dev, sizeof(ErrorLatch), cudaMemcpyDeviceToHost, h->stream));
    FM_CUDA(h, cudaStreamSynchronize(h->stream));
    if (comp) *comp = h->err_host->flag ? h->err_host->comp : -1;
    if (x) *x = h->err_host->flag ? h->err_host->x : -1;
    if (y) *y = h->err_host->flag ? h->err_host->y : -1;
    return FMLBM_OK;
}

fmlbm_status fmlbm_state_size(fmlbm_handle* h, size_t* bytes) {
    if (!h || !bytes) return FMLBM_E_INVALID_ARG;
    size_t gb, g0b, fb;
    buffer_bytes(h->nc, h->lattice, &gb, &g0b, &fb);
    *bytes = sizeof(StateHeader) + gb + g0b + fb;
    return FMLBM_OK;
}

fmlbm_status fmlbm_get_state(fmlbm_handle* h, void* buf, size_t bytes) {
    if (!h || !buf) return FMLBM_E_INVALID_ARG;
    size_t need;
    fmlbm_state_size(h, &need);
    if (bytes < need) return fail(h, FMLBM_E_INVALID_ARG, "state buffer too small");
    size_t gb, g0b, fb;
    buffer_bytes(h->nc, h->lattice, &gb, &g0b, &fb);
    StateHeader hd{kStateMagic, kStateVersion, h->nc, h->lattice.nx, h->lattice.ny, h->lattice.precision,
                   h->step, gb, g0b, fb};
    char* p = static_cast<char*>(buf);
    std::memcpy(p, &hd, sizeof hd);
    p += sizeof hd;
    FM_CUDA(h, cudaMemcpyAsync(p, h->g[h->cur], gb, cudaMemcpyDeviceToHost, h->stream));
    p += gb;
    if (g0b) FM_CUDA(h, cudaMemcpyAsync(p, h->g0[h->cur], g0b, cudaMemcpyDeviceToHost, h->stream));
    p += g0b;
    FM_CUDA(h, cudaMemcpyAsync(p, h->F[h->cur], fb, cudaMemcpyDeviceToHost, h->stream));
    return sync_and_check(h);
}

fmlbm_status fmlbm_set_state(fmlbm_handle* h, const void* buf, size_t bytes) {
    if (!h || !buf || bytes < sizeof(StateHeader)) return FMLBM_E_INVALID_ARG;
    StateHeader hd;
    std::memcpy(&hd, buf, sizeof hd);
    size_t gb, g0b, fb;
    buffer_bytes(h->nc, h->lattice, &gb, &g0b, &fb);
    if (hd.magic != kStateMagic || hd.version != kStateVersion || hd.nc != h->nc || hd.nx != h->lattice.nx ||
        hd.ny != h->lattice.ny || hd.precision != h->lattice.precision || hd.g_bytes != gb ||
        hd.g0_bytes != g0b || hd.f_bytes != fb || bytes < sizeof hd + gb + g0b + fb)
        return fail(h, FMLBM_E_INVALID_ARG, "state does not match this lattice");
    const char* p = static_cast<const char*>(buf) + sizeof hd;
    FM_CUDA(h, cudaMemcpyAsync(h->g[0], p, gb, cudaMemcpyHostToDevice, h->stream));
    p += gb;
    if (g0b) FM_CUDA(h, cudaMemcpyAsync(h->g0[0], p, g0b, cudaMemcpyHostToDevice, h->stream));
    p += g0b;
    FM_CUDA(h, cudaMemcpyAsync(h->F[0], p, fb, cudaMemcpyHostToDevice, h->stream));
    FM_CUDA(h, cudaMemsetAsync(h->err_dev, 0, sizeof(ErrorLatch), h->stream));
    h->cur = 0;
    h->step = hd.step;
    h->have_prev = 0;
    h->pending = -1;  // a request for the replaced state can no longer be served
    for (int k = 0; k < kDiagSlots; ++k)
        if (!h->slot[k].enqueued) h->slot[k].ticket = -1;
    return sync_and_check(h);
}

}  // extern "C"
