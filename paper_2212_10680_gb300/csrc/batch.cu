// Batched lattices (C ABI part of include/fmlbm.h): slots that hold independent
// lattices of one component count and storage precision, advanced together by the
// persistent batch kernel; graph-captured step chunks; per-lattice convergence checks
// and retirement; a tile-shape / grid autotuner.
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "batch.cuh"
#include "fmlbm.h"
#include "fmlbm_internal.h"
#include "fmlbm_launch.cuh"

using namespace fmlbm;

namespace {

struct Slot {
    bool used = false;
    bool active = false;      // stepping
    fmlbm_lattice L{};
    MixConst mc{};
    void* g[2] = {nullptr, nullptr};
    float* g0[2] = {nullptr, nullptr};
    void* F[2] = {nullptr, nullptr};
    void* prev = nullptr;     // density snapshot, storage arithmetic type
    long long steps = 0;      // host mirror of the device counter
    bool have_prev = false;
    double residual = INFINITY;
    double lam[kMaxC] = {};          // phase measure at the last check: mean of ln rho_i
    double phase_change = INFINITY;  // max_i |lam_i| change over the last check interval
    fmlbm_status status = FMLBM_OK;
    size_t bytes = 0;
};

template <int ST>
cudaError_t launch_batch_step_st(int nc, int ty, BatchLattice* lat, const WorkItem* work, int nwork, int grid,
                                 cudaStream_t s);

}  // namespace

struct fmlbm_batch {
    int nc = 0;
    int precision = 0;
    int capacity = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;    // created here (graph capture needs a non-default stream)
    int device = 0, sms = 1;
    std::vector<Slot> slots;
    BatchLattice* d_lat = nullptr;
    std::vector<BatchLattice> h_lat;
    WorkItem* d_work = nullptr;
    int work_cap = 0, nwork = 0;
    bool work_dirty = true;
    int tile_y = kTileYSmall;   // 8-row tiles, 4 blocks per SM: as the single-lattice step
    int grid_mult = 4;          // blocks = grid_mult * SMs (capped by the work count)
    void** d_prev = nullptr;
    double* d_partial = nullptr;
    int partial_cap = 0;
    double* d_out = nullptr;
    double* h_out = nullptr;    // pinned, capacity * (2 nc + 2)
    int criterion = FMLBM_CRITERION_RESIDUAL;
    ErrorLatch* d_err = nullptr;
    ErrorLatch* h_err = nullptr;  // pinned, capacity
    cudaGraphExec_t graph = nullptr;
    int graph_steps = 0;
    size_t bytes_in_use = 0;
    std::string last_error;
};

namespace {

fmlbm_status bfail(fmlbm_batch* b, fmlbm_status s, const std::string& m) {
    if (b) b->last_error = m;
    return s;
}
#define BCUDA(b, call)                                                                            \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return bfail((b), FMLBM_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

size_t rsize(int p) { return p == FMLBM_FP64 ? 8 : 4; }

template <int ST, int NC, int TY>
cudaError_t launch_batch_step_t(BatchLattice* lat, const WorkItem* work, int nwork, int grid, cudaStream_t s) {
    using Real = typename StoreTraits<ST>::Real;
    constexpr size_t smem = sizeof(StepSmem<Real, NC, TY>);
    auto k = batch_step<NC, ST, TY>;
    FMLBM_ENSURE_SMEM(k, smem);
    k<<<grid, dim3(kTX, TY), smem, s>>>(lat, work, nwork);
    return cudaGetLastError();
}

template <int ST, int NC>
cudaError_t launch_batch_step_nc(int ty, BatchLattice* lat, const WorkItem* work, int nwork, int grid, cudaStream_t s) {
    return ty == kTileYLarge ? launch_batch_step_t<ST, NC, kTileYLarge>(lat, work, nwork, grid, s)
                             : launch_batch_step_t<ST, NC, kTileYSmall>(lat, work, nwork, grid, s);
}

template <int ST>
cudaError_t launch_batch_step_st(int nc, int ty, BatchLattice* lat, const WorkItem* work, int nwork, int grid,
                                 cudaStream_t s) {
    switch (nc) {
        case 1: return launch_batch_step_nc<ST, 1>(ty, lat, work, nwork, grid, s);
        case 2: return launch_batch_step_nc<ST, 2>(ty, lat, work, nwork, grid, s);
        case 3: return launch_batch_step_nc<ST, 3>(ty, lat, work, nwork, grid, s);
        case 4: return launch_batch_step_nc<ST, 4>(ty, lat, work, nwork, grid, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_batch_step(const fmlbm_batch* b, int ty, int grid) {
    switch (b->precision) {
        case FMLBM_FP64: return launch_batch_step_st<ST_F64>(b->nc, ty, b->d_lat, b->d_work, b->nwork, grid, b->stream);
        case FMLBM_FP32: return launch_batch_step_st<ST_F32>(b->nc, ty, b->d_lat, b->d_work, b->nwork, grid, b->stream);
        case FMLBM_FP16DEV: return launch_batch_step_st<ST_F16DEV>(b->nc, ty, b->d_lat, b->d_work, b->nwork, grid, b->stream);
        default: return launch_batch_step_st<ST_BF16DEV>(b->nc, ty, b->d_lat, b->d_work, b->nwork, grid, b->stream);
    }
}

template <int ST, int NC>
cudaError_t launch_batch_reduce_nc(const fmlbm_batch* b) {
    batch_reduce<NC, ST><<<b->nwork, dim3(kTX, 8), 0, b->stream>>>(b->d_lat, b->d_work, b->nwork, b->d_prev,
                                                                   b->d_partial);
    const int total = b->capacity * kBatchSums<NC>;
    batch_reduce_final<NC><<<(total + 127) / 128, 128, 0, b->stream>>>(b->d_lat, b->capacity, b->d_partial,
                                                                         b->d_out);
    return cudaGetLastError();
}
template <int ST>
cudaError_t launch_batch_reduce_st(const fmlbm_batch* b) {
    switch (b->nc) {
        case 1: return launch_batch_reduce_nc<ST, 1>(b);
        case 2: return launch_batch_reduce_nc<ST, 2>(b);
        case 3: return launch_batch_reduce_nc<ST, 3>(b);
        case 4: return launch_batch_reduce_nc<ST, 4>(b);
    }
    return cudaErrorInvalidValue;
}
cudaError_t launch_batch_reduce(const fmlbm_batch* b) {
    switch (b->precision) {
        case FMLBM_FP64: return launch_batch_reduce_st<ST_F64>(b);
        case FMLBM_FP32: return launch_batch_reduce_st<ST_F32>(b);
        case FMLBM_FP16DEV: return launch_batch_reduce_st<ST_F16DEV>(b);
        default: return launch_batch_reduce_st<ST_BF16DEV>(b);
    }
}

int grid_for(const fmlbm_batch* b) {
    const int g = b->grid_mult * b->sms;
    return b->nwork < g ? (b->nwork > 0 ? b->nwork : 1) : g;
}

void drop_graph(fmlbm_batch* b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_steps = 0;
}

// Descriptor of slot k (host side), both step parities.
void fill_descriptor(fmlbm_batch* b, int k) {
    Slot& s = b->slots[k];
    BatchLattice& d = b->h_lat[k];
    std::memset(&d, 0, sizeof d);
    if (!s.used) return;
    MixConst mc = s.mc;
    mc.omega = 1.0 / s.L.tau;
    mc.fcoef = 1.0 - 0.5 / s.L.tau;
    mc.invRT = 1.0 / mc.RT;
    for (int p = 0; p < 2; ++p) {
        StepArgs& A = d.args[p];
        A.nx = s.L.nx;
        A.ny = s.L.ny;
        A.stencil = s.L.stencil;
        A.lagged = s.L.velocity_force == FMLBM_FORCE_LAGGED;
        A.gin = s.g[p];
        A.g0in = s.g0[p];
        A.gout = s.g[p ^ 1];
        A.g0out = s.g0[p ^ 1];
        A.Fin = s.F[p];
        A.Fout = s.F[p ^ 1];
        A.err = b->d_err + k;
        A.mixd = mc;
        A.mixf = cast_mix<float>(mc);
    }
    d.step = s.steps;
    d.active = s.active ? 1 : 0;
    d.tile_y = b->tile_y;
}

// Rebuild the work list (active slots only, items of a slot contiguous) and upload the
// descriptors.
fmlbm_status rebuild(fmlbm_batch* b) {
    std::vector<WorkItem> items;
    for (int k = 0; k < b->capacity; ++k) {
        fill_descriptor(b, k);
        Slot& s = b->slots[k];
        BatchLattice& d = b->h_lat[k];
        d.item0 = (int)items.size();
        if (s.used && s.active) {
            for (int y0 = 0; y0 < s.L.ny; y0 += b->tile_y)
                for (int x0 = 0; x0 < s.L.nx; x0 += kTX) items.push_back(WorkItem{k, x0, y0});
        }
        d.nitems = (int)items.size() - d.item0;
    }
    b->nwork = (int)items.size();
    if (b->nwork > b->work_cap) {
        if (b->d_work) cudaFree(b->d_work);
        if (b->d_partial) cudaFree(b->d_partial);
        b->d_work = nullptr;
        b->d_partial = nullptr;
        b->work_cap = b->nwork * 2 + 64;
        BCUDA(b, cudaMalloc((void**)&b->d_work, (size_t)b->work_cap * sizeof(WorkItem)));
        BCUDA(b, cudaMalloc((void**)&b->d_partial, (size_t)b->work_cap * (2 * b->nc + 2) * sizeof(double)));
    }
    if (b->nwork)
        BCUDA(b, cudaMemcpyAsync(b->d_work, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice,
                                 b->stream));
    BCUDA(b, cudaMemcpyAsync(b->d_lat, b->h_lat.data(), (size_t)b->capacity * sizeof(BatchLattice),
                             cudaMemcpyHostToDevice, b->stream));
    std::vector<void*> prev(b->capacity, nullptr);
    for (int k = 0; k < b->capacity; ++k) prev[k] = b->slots[k].prev;
    BCUDA(b, cudaMemcpyAsync(b->d_prev, prev.data(), prev.size() * sizeof(void*), cudaMemcpyHostToDevice, b->stream));
    BCUDA(b, cudaStreamSynchronize(b->stream));  // host vectors above are temporaries
    b->work_dirty = false;
    drop_graph(b);
    return FMLBM_OK;
}

fmlbm_status ensure_work(fmlbm_batch* b) { return b->work_dirty ? rebuild(b) : FMLBM_OK; }

// Enqueue n steps of all active slots (no synchronisation).
fmlbm_status enqueue_steps(fmlbm_batch* b, long long n) {
    const int grid = grid_for(b);
    const int nb = (b->capacity + 127) / 128;
    for (long long k = 0; k < n; ++k) {
        BCUDA(b, launch_batch_step(b, b->tile_y, grid));
        batch_advance<<<nb, 128, 0, b->stream>>>(b->d_lat, b->capacity);
        BCUDA(b, cudaGetLastError());
    }
    for (auto& s : b->slots)
        if (s.used && s.active) s.steps += n;
    return FMLBM_OK;
}

// A chunk of n steps as one CUDA graph (captured once per membership and chunk length).
fmlbm_status run_chunk(fmlbm_batch* b, int n) {
    if (!b->graph || b->graph_steps != n) {
        drop_graph(b);
        cudaGraph_t g = nullptr;
        BCUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        std::vector<long long> saved;
        for (auto& s : b->slots) saved.push_back(s.steps);
        fmlbm_status st = enqueue_steps(b, n);
        for (size_t k = 0; k < saved.size(); ++k) b->slots[k].steps = saved[k];
        cudaError_t e = cudaStreamEndCapture(b->stream, &g);
        if (st != FMLBM_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) return bfail(b, FMLBM_E_CUDA, std::string("capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return bfail(b, FMLBM_E_CUDA, std::string("instantiate: ") + cudaGetErrorString(e));
        b->graph_steps = n;
    }
    BCUDA(b, cudaGraphLaunch(b->graph, b->stream));
    for (auto& s : b->slots)
        if (s.used && s.active) s.steps += n;
    return FMLBM_OK;
}

// Reductions of every active slot -> residuals and phase-measure changes; latched errors ->
// statuses.  Synchronises.
fmlbm_status check_all(fmlbm_batch* b) {
    if (b->nwork == 0) return FMLBM_OK;
    BCUDA(b, launch_batch_reduce(b));
    BCUDA(b, cudaMemcpyAsync(b->h_out, b->d_out, (size_t)b->capacity * (2 * b->nc + 2) * sizeof(double),
                             cudaMemcpyDeviceToHost, b->stream));
    BCUDA(b, cudaMemcpyAsync(b->h_err, b->d_err, (size_t)b->capacity * sizeof(ErrorLatch), cudaMemcpyDeviceToHost,
                             b->stream));
    BCUDA(b, cudaStreamSynchronize(b->stream));
    for (int k = 0; k < b->capacity; ++k) {
        Slot& s = b->slots[k];
        if (!s.used || !s.active) continue;
        const double* o = b->h_out + (size_t)k * (2 * b->nc + 2);
        if (b->h_err[k].flag) {
            s.status = b->h_err[k].flag == 2 ? FMLBM_E_TIMEOUT : FMLBM_E_NONPHYSICAL;
            s.residual = NAN;
            s.phase_change = NAN;
            continue;
        }
        s.residual = s.have_prev ? std::sqrt(o[b->nc]) / std::sqrt(o[b->nc + 1]) : INFINITY;
        const double n = (double)s.L.nx * (double)s.L.ny;
        double change = 0.0;
        for (int i = 0; i < b->nc; ++i) {
            const double lam = o[b->nc + 2 + i] / n;
            // NaN-propagating: a non-finite measure never counts as converged
            const double d = std::fabs(lam - s.lam[i]);
            change = (d > change || d != d) ? d : change;
            s.lam[i] = lam;
        }
        s.phase_change = s.have_prev ? change : INFINITY;
        s.have_prev = true;
    }
    return FMLBM_OK;
}

// The value fmlbm_batch_run compares with tol: the residual or the phase-measure change.
double slot_measure(const fmlbm_batch* b, const Slot& s) {
    return b->criterion == FMLBM_CRITERION_PHASE ? s.phase_change : s.residual;
}

void free_slot(fmlbm_batch* b, Slot& s) {
    for (int p = 0; p < 2; ++p) {
        if (s.g[p]) cudaFreeAsync(s.g[p], b->stream);
        if (s.g0[p]) cudaFreeAsync(s.g0[p], b->stream);
        if (s.F[p]) cudaFreeAsync(s.F[p], b->stream);
    }
    if (s.prev) cudaFreeAsync(s.prev, b->stream);
    b->bytes_in_use -= s.bytes;
    s = Slot();
}

// The moments of a slot's current state into device buffers (rho_out [N][nxy], u_out [2][nxy],
// lnf_out [N][nxy] doubles; u_out and lnf_out may be null), on the batch's stream.
cudaError_t launch_slot_moments(fmlbm_batch* b, int32_t slot, double* rho_out, double* u_out, double* lnf_out) {
    Slot& s = b->slots[slot];
    fill_descriptor(b, slot);
    StepArgs A = b->h_lat[slot].args[s.steps & 1];
    A.rho_out = rho_out;
    A.u_out = u_out;
    A.lnf_out = lnf_out;
    A.gout = nullptr;
    A.g0out = nullptr;
    A.Fout = nullptr;
    const int ty = s.L.ny >= 64 ? kTileYLarge : kTileYSmall;
    switch (b->precision) {
        case FMLBM_FP64: return launch_step<ST_F64>(A, b->nc, true, ty, b->stream);
        case FMLBM_FP32: return launch_step<ST_F32>(A, b->nc, true, ty, b->stream);
        case FMLBM_FP16DEV: return launch_step<ST_F16DEV>(A, b->nc, true, ty, b->stream);
        default: return launch_step<ST_BF16DEV>(A, b->nc, true, ty, b->stream);
    }
}

}  // namespace

extern "C" {

fmlbm_status fmlbm_batch_create(int32_t n_components, int32_t precision, int32_t capacity, void* cuda_stream,
                                fmlbm_batch** out) {
    if (!out || n_components < 1 || n_components > FMLBM_MAX_COMPONENTS || capacity < 1 || capacity > (1 << 20) ||
        precision < FMLBM_FP64 || precision > FMLBM_BF16DEV_LNF64)
        return FMLBM_E_INVALID_ARG;
    // the forms with ln f in double run the single-lattice plain step only
    if (precision == FMLBM_FP16DEV_LNF64 || precision == FMLBM_BF16DEV_LNF64) return FMLBM_E_UNSUPPORTED;
    *out = nullptr;
    fmlbm_batch* b = new (std::nothrow) fmlbm_batch();
    if (!b) return FMLBM_E_OOM;
    b->nc = n_components;
    b->precision = precision;
    b->capacity = capacity;
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    if (!b->stream) {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete b;
            return FMLBM_E_CUDA;
        }
        b->own_stream = true;
    }
    b->slots.resize(capacity);
    b->h_lat.resize(capacity);
    bool ok = cudaGetDevice(&b->device) == cudaSuccess &&
              cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device) == cudaSuccess;
    ok = ok && cudaMalloc((void**)&b->d_lat, (size_t)capacity * sizeof(BatchLattice)) == cudaSuccess;
    ok = ok && cudaMalloc((void**)&b->d_prev, (size_t)capacity * sizeof(void*)) == cudaSuccess;
    ok = ok && cudaMalloc((void**)&b->d_out, (size_t)capacity * (2 * n_components + 2) * sizeof(double)) == cudaSuccess;
    ok = ok && cudaMalloc((void**)&b->d_err, (size_t)capacity * sizeof(ErrorLatch)) == cudaSuccess;
    ok = ok && cudaMallocHost((void**)&b->h_out, (size_t)capacity * (2 * n_components + 2) * sizeof(double)) == cudaSuccess;
    ok = ok && cudaMallocHost((void**)&b->h_err, (size_t)capacity * sizeof(ErrorLatch)) == cudaSuccess;
    ok = ok && cudaMemsetAsync(b->d_err, 0, (size_t)capacity * sizeof(ErrorLatch), b->stream) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        fmlbm_batch_destroy(b);
        return FMLBM_E_OOM;
    }
    *out = b;
    return FMLBM_OK;
}

void fmlbm_batch_destroy(fmlbm_batch* b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    drop_graph(b);
    for (auto& s : b->slots)
        if (s.used) free_slot(b, s);
    cudaStreamSynchronize(b->stream);
    if (b->d_lat) cudaFree(b->d_lat);
    if (b->d_work) cudaFree(b->d_work);
    if (b->d_prev) cudaFree(b->d_prev);
    if (b->d_partial) cudaFree(b->d_partial);
    if (b->d_out) cudaFree(b->d_out);
    if (b->d_err) cudaFree(b->d_err);
    if (b->h_out) cudaFreeHost(b->h_out);
    if (b->h_err) cudaFreeHost(b->h_err);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
}

const char* fmlbm_batch_last_error(const fmlbm_batch* b) { return b ? b->last_error.c_str() : ""; }

fmlbm_status fmlbm_batch_add(fmlbm_batch* b, const fmlbm_mixture* mixture, const fmlbm_lattice* lattice,
                             const double* rho_host, int32_t* slot_out) {
    if (!b || !mixture || !lattice || !rho_host || !slot_out) return bfail(b, FMLBM_E_INVALID_ARG, "null argument");
    if (mixture->n_components != b->nc) return bfail(b, FMLBM_E_INVALID_ARG, "component count differs from the batch");
    if (lattice->precision != b->precision) return bfail(b, FMLBM_E_INVALID_ARG, "precision differs from the batch");
    if (lattice->formulation != FMLBM_WELL_BALANCED)
        return bfail(b, FMLBM_E_INVALID_ARG, "batches run the well-balanced formulation only");
    std::string why;
    MixConst mc;
    if (!fmlbm_internal_mixture_constants(*mixture, &mc, &why) ||
        !fmlbm_internal_lattice_ok(*lattice, b->nc, &why))
        return bfail(b, FMLBM_E_INVALID_ARG, why);
    int k = -1;
    for (int q = 0; q < b->capacity; ++q)
        if (!b->slots[q].used) {
            k = q;
            break;
        }
    if (k < 0) return bfail(b, FMLBM_E_BUSY, "no free slot");
    Slot s;
    s.used = true;
    s.L = *lattice;
    s.mc = mc;
    const size_t nxy = (size_t)lattice->nx * lattice->ny;
    const bool dev16 = b->precision == FMLBM_FP16DEV || b->precision == FMLBM_BF16DEV;
    const size_t gb = dev16 ? (size_t)b->nc * 8 * nxy * 2 : (size_t)b->nc * 9 * nxy * rsize(b->precision);
    const size_t g0b = dev16 ? (size_t)b->nc * nxy * 4 : 0;
    const size_t fb = 2 * nxy * rsize(b->precision);
    const size_t pb = (size_t)b->nc * nxy * rsize(b->precision);
    bool ok = true;
    for (int p = 0; p < 2 && ok; ++p) {
        ok = ok && cudaMallocAsync(&s.g[p], gb, b->stream) == cudaSuccess;
        if (g0b) ok = ok && cudaMallocAsync((void**)&s.g0[p], g0b, b->stream) == cudaSuccess;
        ok = ok && cudaMallocAsync(&s.F[p], fb, b->stream) == cudaSuccess;
    }
    ok = ok && cudaMallocAsync(&s.prev, pb, b->stream) == cudaSuccess;
    s.bytes = 2 * (gb + g0b + fb) + pb;
    b->bytes_in_use += s.bytes;
    if (!ok) {
        cudaGetLastError();
        free_slot(b, s);
        return bfail(b, FMLBM_E_OOM, "device allocation failed");
    }
    // initialise: fluid at rest from the host densities, into buffer 0
    double* d = nullptr;
    const size_t rb = (size_t)b->nc * nxy * sizeof(double);
    cudaError_t e = cudaMallocAsync((void**)&d, rb, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d, rho_host, rb, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) {
        StepArgs A;
        std::memset(&A, 0, sizeof A);
        A.nx = lattice->nx;
        A.ny = lattice->ny;
        A.gout = s.g[0];
        A.g0out = s.g0[0];
        A.Fout = s.F[0];
        switch (b->precision) {
            case FMLBM_FP64: e = launch_init<ST_F64>(A, b->nc, d, b->stream); break;
            case FMLBM_FP32: e = launch_init<ST_F32>(A, b->nc, d, b->stream); break;
            case FMLBM_FP16DEV: e = launch_init<ST_F16DEV>(A, b->nc, d, b->stream); break;
            default: e = launch_init<ST_BF16DEV>(A, b->nc, d, b->stream); break;
        }
    }
    if (d) cudaFreeAsync(d, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_err + k, 0, sizeof(ErrorLatch), b->stream);
    if (e != cudaSuccess) {
        free_slot(b, s);
        return bfail(b, FMLBM_E_CUDA, std::string("batch add: ") + cudaGetErrorString(e));
    }
    s.active = true;
    b->slots[k] = s;
    b->work_dirty = true;
    *slot_out = k;
    return FMLBM_OK;
}

fmlbm_status fmlbm_batch_remove(fmlbm_batch* b, int32_t slot) {
    if (!b || slot < 0 || slot >= b->capacity || !b->slots[slot].used) return bfail(b, FMLBM_E_INVALID_ARG, "bad slot");
    BCUDA(b, cudaStreamSynchronize(b->stream));
    free_slot(b, b->slots[slot]);
    b->work_dirty = true;
    return FMLBM_OK;
}

fmlbm_status fmlbm_batch_set_active(fmlbm_batch* b, int32_t slot, int32_t active) {
    if (!b || slot < 0 || slot >= b->capacity || !b->slots[slot].used) return bfail(b, FMLBM_E_INVALID_ARG, "bad slot");
    if (b->slots[slot].active != (active != 0)) {
        b->slots[slot].active = active != 0;
        b->work_dirty = true;
    }
    return FMLBM_OK;
}

fmlbm_status fmlbm_batch_step(fmlbm_batch* b, int64_t nsteps) {
    if (!b || nsteps < 0) return bfail(b, FMLBM_E_INVALID_ARG, "bad argument");
    fmlbm_status s = ensure_work(b);
    if (s != FMLBM_OK || b->nwork == 0) return s;
    return enqueue_steps(b, nsteps);
}

fmlbm_status fmlbm_batch_run(fmlbm_batch* b, int64_t max_steps, int32_t check_every, double tol, int64_t* steps_out,
                             double* residual_out, int32_t* status_out) {
    if (!b || max_steps < 0 || check_every < 1) return bfail(b, FMLBM_E_INVALID_ARG, "bad argument");
    fmlbm_status st = ensure_work(b);
    if (st != FMLBM_OK) return st;
    // first snapshot of every active slot
    st = check_all(b);
    if (st != FMLBM_OK) return st;
    while (true) {
        bool any = false;
        for (auto& s : b->slots)
            if (s.used && s.active) any = true;
        if (!any) break;
        long long done_min = -1;
        for (auto& s : b->slots)
            if (s.used && s.active) done_min = done_min < 0 ? s.steps : std::min(done_min, s.steps);
        const long long left = max_steps - done_min;
        const int n = (int)std::min<long long>(check_every, std::max<long long>(left, 1));
        st = ensure_work(b);
        if (st != FMLBM_OK) return st;
        st = run_chunk(b, n);
        if (st != FMLBM_OK) return st;
        st = check_all(b);
        if (st != FMLBM_OK) return st;
        for (auto& s : b->slots) {
            if (!s.used || !s.active) continue;
            bool retire = false;
            if (s.status != FMLBM_OK) retire = true;
            else if (slot_measure(b, s) < tol) retire = true;
            else if (s.steps >= max_steps) {
                s.status = FMLBM_E_NOT_CONVERGED;
                retire = true;
            }
            if (retire) {
                s.active = false;
                b->work_dirty = true;
            }
        }
    }
    for (int k = 0; k < b->capacity; ++k) {
        const Slot& s = b->slots[k];
        if (steps_out) steps_out[k] = s.used ? s.steps : 0;
        if (residual_out) residual_out[k] = s.used ? slot_measure(b, s) : NAN;
        if (status_out) status_out[k] = s.used ? s.status : FMLBM_E_INVALID_ARG;
    }
    return FMLBM_OK;
}

fmlbm_status fmlbm_batch_run_chunk(fmlbm_batch* b, int32_t steps) {
    if (!b || steps < 1) return bfail(b, FMLBM_E_INVALID_ARG, "bad argument");
    fmlbm_status st = ensure_work(b);
    if (st != FMLBM_OK || b->nwork == 0) return st;
    st = run_chunk(b, steps);
    if (st != FMLBM_OK) return st;
    return check_all(b);
}

fmlbm_status fmlbm_batch_slot_info(fmlbm_batch* b, int32_t slot, int64_t* steps, double* residual, int32_t* status,
                                   int32_t* active) {
    if (!b || slot < 0 || slot >= b->capacity || !b->slots[slot].used) return bfail(b, FMLBM_E_INVALID_ARG, "bad slot");
    const Slot& s = b->slots[slot];
    if (steps) *steps = s.steps;
    if (residual) *residual = s.residual;
    if (status) *status = s.status;
    if (active) *active = s.active ? 1 : 0;
    return FMLBM_OK;
}

fmlbm_status fmlbm_batch_slot_phase_change(fmlbm_batch* b, int32_t slot, double* change) {
    if (!b || !change || slot < 0 || slot >= b->capacity || !b->slots[slot].used)
        return bfail(b, FMLBM_E_INVALID_ARG, "bad slot");
    *change = b->slots[slot].phase_change;
    return FMLBM_OK;
}

fmlbm_status fmlbm_batch_set_criterion(fmlbm_batch* b, int32_t criterion) {
    if (!b || (criterion != FMLBM_CRITERION_RESIDUAL && criterion != FMLBM_CRITERION_PHASE))
        return bfail(b, FMLBM_E_INVALID_ARG, "unknown convergence criterion");
    b->criterion = criterion;
    return FMLBM_OK;
}

fmlbm_status fmlbm_batch_check(fmlbm_batch* b) {
    if (!b) return FMLBM_E_INVALID_ARG;
    fmlbm_status st = ensure_work(b);
    if (st != FMLBM_OK) return st;
    return check_all(b);
}

fmlbm_status fmlbm_batch_moments(fmlbm_batch* b, int32_t slot, double* rho, double* u, double* lnf) {
    if (!b || slot < 0 || slot >= b->capacity || !b->slots[slot].used) return bfail(b, FMLBM_E_INVALID_ARG, "bad slot");
    Slot& s = b->slots[slot];
    const size_t nxy = (size_t)s.L.nx * s.L.ny;
    const size_t fb = (size_t)b->nc * nxy * sizeof(double);
    double* d = nullptr;
    BCUDA(b, cudaMallocAsync((void**)&d, 2 * fb + 2 * nxy * sizeof(double), b->stream));
    cudaError_t e = launch_slot_moments(b, slot, d, d + 2 * (size_t)b->nc * nxy, d + (size_t)b->nc * nxy);
    if (e == cudaSuccess && rho) e = cudaMemcpyAsync(rho, d, fb, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess && lnf) e = cudaMemcpyAsync(lnf, d + (size_t)b->nc * nxy, fb, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess && u)
        e = cudaMemcpyAsync(u, d + 2 * (size_t)b->nc * nxy, 2 * nxy * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    cudaFreeAsync(d, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, FMLBM_E_CUDA, std::string("batch moments: ") + cudaGetErrorString(e));
    return FMLBM_OK;
}

fmlbm_status fmlbm_batch_phases(fmlbm_batch* b, int32_t slot, double* rho_liquid, double* rho_vapour) {
    if (!b || slot < 0 || slot >= b->capacity || !b->slots[slot].used) return bfail(b, FMLBM_E_INVALID_ARG, "bad slot");
    Slot& s = b->slots[slot];
    const size_t nxy = (size_t)s.L.nx * s.L.ny;
    double* d = nullptr;
    BCUDA(b, cudaMallocAsync((void**)&d, ((size_t)b->nc * nxy + 2 * kMaxC) * sizeof(double), b->stream));
    double* out = d + (size_t)b->nc * nxy;
    cudaError_t e = launch_slot_moments(b, slot, d, nullptr, nullptr);
    if (e == cudaSuccess) {
        const MixConst& m = b->h_lat[slot].args[0].mixd;
        switch (b->nc) {
            case 1: phase_nodes<1><<<1, kPhaseThreads, 0, b->stream>>>(d, s.L.nx, s.L.ny, m, out); break;
            case 2: phase_nodes<2><<<1, kPhaseThreads, 0, b->stream>>>(d, s.L.nx, s.L.ny, m, out); break;
            case 3: phase_nodes<3><<<1, kPhaseThreads, 0, b->stream>>>(d, s.L.nx, s.L.ny, m, out); break;
            default: phase_nodes<4><<<1, kPhaseThreads, 0, b->stream>>>(d, s.L.nx, s.L.ny, m, out); break;
        }
        e = cudaGetLastError();
    }
    double h[2 * kMaxC];
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, out, 2 * b->nc * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    cudaFreeAsync(d, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, FMLBM_E_CUDA, std::string("batch phases: ") + cudaGetErrorString(e));
    for (int i = 0; i < b->nc; ++i) {
        if (rho_liquid) rho_liquid[i] = h[i];
        if (rho_vapour) rho_vapour[i] = h[b->nc + i];
    }
    return FMLBM_OK;
}

fmlbm_status fmlbm_batch_get_distributions(fmlbm_batch* b, int32_t slot, double* g, double* force) {
    if (!b || slot < 0 || slot >= b->capacity || !b->slots[slot].used) return bfail(b, FMLBM_E_INVALID_ARG, "bad slot");
    Slot& s = b->slots[slot];
    fill_descriptor(b, slot);
    const StepArgs A = b->h_lat[slot].args[s.steps & 1];
    const size_t nxy = (size_t)s.L.nx * s.L.ny;
    cudaError_t e = cudaSuccess;
    if (g) {
        const size_t gbytes = (size_t)b->nc * 9 * nxy * sizeof(double);
        double* d = nullptr;
        BCUDA(b, cudaMallocAsync((void**)&d, gbytes, b->stream));
        switch (b->precision) {
            case FMLBM_FP64: e = launch_convert<ST_F64>(A, b->nc, nullptr, d, false, b->stream); break;
            case FMLBM_FP32: e = launch_convert<ST_F32>(A, b->nc, nullptr, d, false, b->stream); break;
            case FMLBM_FP16DEV: e = launch_convert<ST_F16DEV>(A, b->nc, nullptr, d, false, b->stream); break;
            default: e = launch_convert<ST_BF16DEV>(A, b->nc, nullptr, d, false, b->stream); break;
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(g, d, gbytes, cudaMemcpyDeviceToHost, b->stream);
        cudaFreeAsync(d, b->stream);
    }
    if (e == cudaSuccess && force) {
        std::vector<float> tmp;
        if (b->precision == FMLBM_FP64) {
            e = cudaMemcpyAsync(force, A.Fin, 2 * nxy * 8, cudaMemcpyDeviceToHost, b->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        } else {
            tmp.resize(2 * nxy);
            e = cudaMemcpyAsync(tmp.data(), A.Fin, 2 * nxy * 4, cudaMemcpyDeviceToHost, b->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
            for (size_t k = 0; k < tmp.size() && e == cudaSuccess; ++k) force[k] = tmp[k];
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, FMLBM_E_CUDA, std::string("batch distributions: ") + cudaGetErrorString(e));
    return FMLBM_OK;
}

fmlbm_status fmlbm_batch_autotune(fmlbm_batch* b, int32_t steps_per_trial, int32_t* tile_y_out, int32_t* blocks_out,
                                  double* ms_per_step_out) {
    if (!b || steps_per_trial < 1) return bfail(b, FMLBM_E_INVALID_ARG, "bad argument");
    const int tys[2] = {kTileYSmall, kTileYLarge};
    const int mults[4] = {1, 2, 4, 8};
    float best = 1e30f;
    int best_ty = b->tile_y, best_mult = b->grid_mult;
    cudaEvent_t e0, e1;
    BCUDA(b, cudaEventCreate(&e0));
    BCUDA(b, cudaEventCreate(&e1));
    for (int ty : tys) {
        b->tile_y = ty;
        b->work_dirty = true;
        fmlbm_status st = ensure_work(b);
        if (st != FMLBM_OK) return st;
        if (b->nwork == 0) break;
        for (int mult : mults) {
            b->grid_mult = mult;
            // each trial advances the lattices by real steps: the tiling does not change results
            st = enqueue_steps(b, 1);
            if (st != FMLBM_OK) return st;
            BCUDA(b, cudaEventRecord(e0, b->stream));
            st = enqueue_steps(b, steps_per_trial);
            if (st != FMLBM_OK) return st;
            BCUDA(b, cudaEventRecord(e1, b->stream));
            BCUDA(b, cudaEventSynchronize(e1));
            float ms = 0.f;
            BCUDA(b, cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) {
                best = ms;
                best_ty = ty;
                best_mult = mult;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->tile_y = best_ty;
    b->grid_mult = best_mult;
    b->work_dirty = true;
    if (tile_y_out) *tile_y_out = best_ty;
    if (blocks_out) *blocks_out = best_mult * b->sms;
    if (ms_per_step_out) *ms_per_step_out = best / steps_per_trial;
    return FMLBM_OK;
}

fmlbm_status fmlbm_batch_bytes(fmlbm_batch* b, size_t* bytes) {
    if (!b || !bytes) return FMLBM_E_INVALID_ARG;
    *bytes = b->bytes_in_use;
    return FMLBM_OK;
}

}  // extern "C"
