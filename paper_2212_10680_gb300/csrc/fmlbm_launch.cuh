// Host-side launchers of the device kernels, one explicit instantiation set per
// storage precision (step_f64.cu, step_f32.cu, step_f16.cu, step_bf16.cu).
#pragma once

#include <atomic>

#include "fmlbm_multi.cuh"
#include "fmlbm_pair.cuh"
#include "fmlbm_tma.cuh"

namespace fmlbm {

// The dynamic shared-memory limit of a kernel is a property of each device, and launches
// come from any thread (a server's worker and its callers).  Each kernel keeps one atomic
// bit mask of the devices it has been raised on (bit = device ordinal; ordinals from 64 on
// raise it at every launch).  Two threads racing both set the same value: harmless.
inline cudaError_t ensure_smem_attr(std::atomic<unsigned long long>& done, const void* func, size_t bytes) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = dev >= 0 && dev < 64 ? 1ull << dev : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_release);
    return e;
}
#define FMLBM_ENSURE_SMEM(kernel, bytes)                                                     \
    do {                                                                                   \
        static std::atomic<unsigned long long> done_{0ull};                                \
        cudaError_t e_ = ensure_smem_attr(done_, reinterpret_cast<const void*>(kernel), (bytes)); \
        if (e_ != cudaSuccess) return e_;                                                  \
    } while (0)

// Tile heights of the fused step (tile width is one warp).  The host picks one per
// lattice (fmlbm_set_tile_height / the batch autotuner).
constexpr int kTileYSmall = 8;
constexpr int kTileYLarge = 16;
constexpr int kTileYHuge = 32;

template <int ST>
cudaError_t launch_step(const StepArgs& A, int nc, bool moments, int tile_y, cudaStream_t s);
// Persistent TMA-fed step (float and 16-bit storage); maps[0]: float planes, maps[1]:
// 16-bit planes (deviation forms).  tma_ok = 0 sends every tile down the plain pull path.
// single_stage = false: persistent double-buffered blocks (one per SM);
// true: one tile per block, single stage, as many blocks per SM as shared memory admits.
template <int ST>
cudaError_t launch_step_tma(const StepArgs& A, int nc, const CUtensorMap* maps, int tma_ok, bool single_stage,
                            cudaStream_t s);
// Whether the TMA variant exists for this storage and component count (shared memory).
template <int ST>
bool tma_supported(int nc);
// The paired step (two nodes per thread, packed float arithmetic; float and 16-bit
// storage, well-balanced formulation).  cudaErrorNotSupported for FP64 storage.
template <int ST>
cudaError_t launch_step_pair(const StepArgs& A, int nc, cudaStream_t s);
template <int ST>
bool pair_supported(int nc);
// K time steps in one cooperative launch of the multi-step kernel (fmlbm_multi.cuh): A0 the
// arguments of the first step (reading the current buffer), A1 those of the second.  done:
// at least multi_tiles(nx, ny) counters of device scratch (reset here, on the stream).
// Float and 16-bit storage, the specialised options only (spec_options); otherwise
// cudaErrorNotSupported.
template <int ST>
cudaError_t launch_steps_multi(const StepArgs& A0, const StepArgs& A1, int nc, int nsteps, long long* done,
                               cudaStream_t s);
inline int multi_tiles(int nx, int ny) { return ((nx + kTX - 1) / kTX) * ((ny + kTileYSmall - 1) / kTileYSmall); }

template <int ST>
cudaError_t launch_init(const StepArgs& A, int nc, const double* rho, cudaStream_t s);
template <int ST>
cudaError_t launch_convert(const StepArgs& A, int nc, const double* gin_d, double* gout_d, bool to_storage,
                           cudaStream_t s);
// rho_prev: NC * nx * ny values of the storage arithmetic type (double for FP64, else float);
// partial: (NC + 2) * reduce_blocks(nx, ny) doubles.
template <int ST>
cudaError_t launch_reduce(const StepArgs& A, int nc, void* rho_prev, int have_prev, void* partial,
                          double* out, cudaStream_t s);

// Phase measure: out[i] = sum over the nodes of ln rho_i (NC doubles, device); partial:
// NC * reduce_blocks(nx, ny) doubles.
template <int ST>
cudaError_t launch_lnrho(const StepArgs& A, int nc, double* partial, double* out, cudaStream_t s);

// The fixed-order final sum alone, for partial sums a fused step wrote (A.diag_partial):
// (NC + 2) doubles per 32 x 8 strip; latch (may be null): copied to out + kMaxC + 2.
inline cudaError_t launch_reduce_final(int nc, const void* partial, int nx, int ny, double* out, cudaStream_t s,
                                       const ErrorLatch* latch = nullptr) {
    const int nb = reduce_blocks(nx, ny);
    const double* p = static_cast<const double*>(partial);
    switch (nc) {
        case 1: reduce_final<1><<<1 + 2, kFinalThreads, 0, s>>>(p, nb, out, latch); break;
        case 2: reduce_final<2><<<2 + 2, kFinalThreads, 0, s>>>(p, nb, out, latch); break;
        case 3: reduce_final<3><<<3 + 2, kFinalThreads, 0, s>>>(p, nb, out, latch); break;
        case 4: reduce_final<4><<<4 + 2, kFinalThreads, 0, s>>>(p, nb, out, latch); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// The specialised step (fused_step<..., SPEC = true>): float and 16-bit storage, 8-row tiles,
// for lattices with the Peng-Robinson EOS, isotropic stencils, the lagged velocity reading and
// the well-balanced formulation.
template <int ST> constexpr bool kSpecStep = ST == ST_F32 || ST == ST_F16DEV || ST == ST_BF16DEV;
inline bool spec_options(const StepArgs& A) {
    return A.mixd.eos == 0 && A.stencil == 0 && A.lagged != 0 && A.standard == 0;
}

#define FMLBM_DEFINE_LAUNCHERS(ST)                                                                        \
    template <int NC, bool MOM, int TY, bool STD = false, bool SPEC = false>                              \
    static cudaError_t launch_step_nc_##ST(const StepArgs& A, cudaStream_t s) {                           \
        using Real = typename StoreTraits<ST>::Real;                                                      \
        /* + the parked values and the diagnostics snapshot copy of the tile's nodes */                 \
        constexpr size_t smem = sizeof(StepSmem<Real, NC, TY>) + park_bytes<NC, ST, TY>() +                \
                                (MOM ? 0 : (size_t)NC * TY * kTX * sizeof(Real));                         \
        auto k = fused_step<NC, ST, TY, MOM, STD, SPEC>;                                                  \
        FMLBM_ENSURE_SMEM(k, smem);                                                                       \
        dim3 grid((A.nx + kTX - 1) / kTX, (A.ny + TY - 1) / TY);                                          \
        const Planes P = make_planes(A, NC, kDev16<ST>,                                                   \
                                     ST == ST_F64 ? 8 : (ST == ST_F32 ? 4 : 2));                          \
        k<<<grid, dim3(kTX, TY), smem, s>>>(A, P);                                                        \
        return cudaGetLastError();                                                                        \
    }                                                                                                     \
    template <int NC>                                                                                     \
    static cudaError_t launch_step_ty_##ST(const StepArgs& A, bool moments, int tile_y, cudaStream_t s) { \
        /* the standard formulation: FP64 and FP32 storage, 8-row tiles */                              \
        if constexpr (ST == ST_F64 || ST == ST_F32) {                                                     \
            if (A.standard)                                                                               \
                return moments ? launch_step_nc_##ST<NC, true, kTileYSmall, true>(A, s)                   \
                               : launch_step_nc_##ST<NC, false, kTileYSmall, true>(A, s);                 \
        } else {                                                                                          \
            if (A.standard) return cudaErrorNotSupported;                                                 \
        }                                                                                                 \
        if (tile_y == kTileYLarge)                                                                        \
            return moments ? launch_step_nc_##ST<NC, true, kTileYLarge>(A, s)                             \
                           : launch_step_nc_##ST<NC, false, kTileYLarge>(A, s);                           \
        if (tile_y == kTileYHuge && !moments) return launch_step_nc_##ST<NC, false, kTileYHuge>(A, s);    \
        if constexpr (kSpecStep<ST>) {                                                                    \
            if (!moments && spec_options(A)) return launch_step_nc_##ST<NC, false, kTileYSmall, false, true>(A, s); \
        }                                                                                                 \
        return moments ? launch_step_nc_##ST<NC, true, kTileYSmall>(A, s)                                 \
                       : launch_step_nc_##ST<NC, false, kTileYSmall>(A, s);                               \
    }                                                                                                     \
    template <>                                                                                           \
    cudaError_t launch_step<ST>(const StepArgs& A, int nc, bool moments, int tile_y, cudaStream_t s) {    \
        switch (nc) {                                                                                     \
            case 1: return launch_step_ty_##ST<1>(A, moments, tile_y, s);                                 \
            case 2: return launch_step_ty_##ST<2>(A, moments, tile_y, s);                                 \
            case 3: return launch_step_ty_##ST<3>(A, moments, tile_y, s);                                 \
            case 4: return launch_step_ty_##ST<4>(A, moments, tile_y, s);                                 \
        }                                                                                                 \
        return cudaErrorInvalidValue;                                                                     \
    }                                                                                                     \
    static int grid_1d(size_t n) {                                                                        \
        size_t b = (n + 255) / 256;                                                                       \
        return (int)(b > 4096 ? 4096 : (b == 0 ? 1 : b));                                                 \
    }                                                                                                     \
    template <>                                                                                           \
    cudaError_t launch_init<ST>(const StepArgs& A, int nc, const double* rho, cudaStream_t s) {           \
        const int g = grid_1d((size_t)A.nx * A.ny);                                                       \
        switch (nc) {                                                                                     \
            case 1: init_rest<1, ST><<<g, 256, 0, s>>>(A, rho); break;                                    \
            case 2: init_rest<2, ST><<<g, 256, 0, s>>>(A, rho); break;                                    \
            case 3: init_rest<3, ST><<<g, 256, 0, s>>>(A, rho); break;                                    \
            case 4: init_rest<4, ST><<<g, 256, 0, s>>>(A, rho); break;                                    \
            default: return cudaErrorInvalidValue;                                                        \
        }                                                                                                 \
        return cudaGetLastError();                                                                        \
    }                                                                                                     \
    template <>                                                                                           \
    cudaError_t launch_convert<ST>(const StepArgs& A, int nc, const double* gin_d, double* gout_d,        \
                                   bool to_storage, cudaStream_t s) {                                     \
        const int g = grid_1d((size_t)A.nx * A.ny);                                                       \
        switch (nc) {                                                                                     \
            case 1: convert_g<1, ST><<<g, 256, 0, s>>>(A, gin_d, gout_d, to_storage); break;              \
            case 2: convert_g<2, ST><<<g, 256, 0, s>>>(A, gin_d, gout_d, to_storage); break;              \
            case 3: convert_g<3, ST><<<g, 256, 0, s>>>(A, gin_d, gout_d, to_storage); break;              \
            case 4: convert_g<4, ST><<<g, 256, 0, s>>>(A, gin_d, gout_d, to_storage); break;              \
            default: return cudaErrorInvalidValue;                                                        \
        }                                                                                                 \
        return cudaGetLastError();                                                                        \
    }                                                                                                     \
    template <int NC>                                                                                     \
    static cudaError_t launch_reduce_nc_##ST(const StepArgs& A, void* rho_prev, int have_prev,            \
                                             void* partial, double* out, cudaStream_t s) {                \
        using Real = typename StoreTraits<ST>::Real;                                                      \
        dim3 grid((A.nx + kTX - 1) / kTX, (A.ny + kRedTY - 1) / kRedTY);                                  \
        reduce_partial<NC, ST><<<grid, dim3(kTX, kRedTY), 0, s>>>(A, static_cast<Real*>(rho_prev),        \
                                                                   have_prev, static_cast<double*>(partial)); \
        reduce_final<NC><<<NC + 2, kFinalThreads, 0, s>>>(static_cast<const double*>(partial),             \
                                                          reduce_blocks(A.nx, A.ny), out, A.err);         \
        return cudaGetLastError();                                                                        \
    }                                                                                                     \
    template <>                                                                                           \
    cudaError_t launch_reduce<ST>(const StepArgs& A, int nc, void* rho_prev, int have_prev,               \
                                  void* partial, double* out, cudaStream_t s) {                           \
        switch (nc) {                                                                                     \
            case 1: return launch_reduce_nc_##ST<1>(A, rho_prev, have_prev, partial, out, s);             \
            case 2: return launch_reduce_nc_##ST<2>(A, rho_prev, have_prev, partial, out, s);             \
            case 3: return launch_reduce_nc_##ST<3>(A, rho_prev, have_prev, partial, out, s);             \
            case 4: return launch_reduce_nc_##ST<4>(A, rho_prev, have_prev, partial, out, s);             \
        }                                                                                                 \
        return cudaErrorInvalidValue;                                                                     \
    }                                                                                                     \
    template <int NC>                                                                                     \
    static cudaError_t launch_lnrho_nc_##ST(const StepArgs& A, double* partial, double* out,              \
                                            cudaStream_t s) {                                             \
        dim3 grid((A.nx + kTX - 1) / kTX, (A.ny + kRedTY - 1) / kRedTY);                                  \
        lnrho_partial<NC, ST><<<grid, dim3(kTX, kRedTY), 0, s>>>(A, partial);                             \
        sum_columns<NC><<<NC, kFinalThreads, 0, s>>>(partial, reduce_blocks(A.nx, A.ny), out);            \
        return cudaGetLastError();                                                                        \
    }                                                                                                     \
    template <>                                                                                           \
    cudaError_t launch_lnrho<ST>(const StepArgs& A, int nc, double* partial, double* out, cudaStream_t s) { \
        switch (nc) {                                                                                     \
            case 1: return launch_lnrho_nc_##ST<1>(A, partial, out, s);                                   \
            case 2: return launch_lnrho_nc_##ST<2>(A, partial, out, s);                                   \
            case 3: return launch_lnrho_nc_##ST<3>(A, partial, out, s);                                   \
            case 4: return launch_lnrho_nc_##ST<4>(A, partial, out, s);                                   \
        }                                                                                                 \
        return cudaErrorInvalidValue;                                                                     \
    }

#define FMLBM_DEFINE_TMA_LAUNCHER(ST)                                                                     \
    template <int NC, bool SINGLE>                                                                        \
    static cudaError_t launch_tma_nc_##ST(const StepArgs& A, const CUtensorMap* maps, int tma_ok,         \
                                          cudaStream_t s) {                                               \
        using L = TmaLayout<NC, ST, kTmaTileY>;                                                           \
        if constexpr (!L::fits) {                                                                         \
            return cudaErrorNotSupported;                                                                 \
        } else {                                                                                          \
            constexpr int NS = SINGLE ? 1 : L::stages;                                                    \
            /* single stage: as many blocks as shared memory admits (at most 4), which */             \
            /* also bounds the registers the compiler may give each thread              */             \
            constexpr size_t smem1 = L::scratch_bytes + L::stage_bytes + 64 + 1024;                     \
            constexpr int fit1 = (int)((228 * 1024) / smem1);                                          \
            constexpr int MINB = SINGLE ? (fit1 > 4 ? 4 : (fit1 < 1 ? 1 : fit1)) : 1;                \
            constexpr size_t smem = L::scratch_bytes + NS * L::stage_bytes + 64;                          \
            auto k = fused_step_tma<NC, ST, kTmaTileY, NS, MINB>;                                         \
            FMLBM_ENSURE_SMEM(k, smem);                                                                   \
            /* blocks per SM and SM count of the current device (per device: a process may */          \
            /* drive several; computed at each launch of the persistent form only)          */          \
            int per_sm = 1, sms = 1;                                                                      \
            if (!SINGLE) {                                                                                \
                int dev = 0;                                                                              \
                cudaError_t e = cudaGetDevice(&dev);                                                      \
                if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev); \
                if (e == cudaSuccess)                                                                     \
                    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kTX * kTmaTileY, smem); \
                if (e != cudaSuccess) return e;                                                           \
                if (per_sm < 1) return cudaErrorInvalidConfiguration;                                     \
            }                                                                                             \
            const int ntiles = ((A.nx + kTX - 1) / kTX) * ((A.ny + kTmaTileY - 1) / kTmaTileY);           \
            const int grid = SINGLE ? ntiles : (ntiles < sms * per_sm ? ntiles : sms * per_sm);           \
            k<<<grid, dim3(kTX, kTmaTileY), smem, s>>>(A, maps[0], maps[1], tma_ok);                      \
            return cudaGetLastError();                                                                    \
        }                                                                                                 \
    }                                                                                                     \
    template <int NC>                                                                                     \
    static cudaError_t launch_tma_mode_##ST(const StepArgs& A, const CUtensorMap* maps, int tma_ok,       \
                                            bool single, cudaStream_t s) {                                \
        return single ? launch_tma_nc_##ST<NC, true>(A, maps, tma_ok, s)                                  \
                      : launch_tma_nc_##ST<NC, false>(A, maps, tma_ok, s);                                \
    }                                                                                                     \
    template <>                                                                                           \
    cudaError_t launch_step_tma<ST>(const StepArgs& A, int nc, const CUtensorMap* maps, int tma_ok,       \
                                    bool single, cudaStream_t s) {                                        \
        switch (nc) {                                                                                     \
            case 1: return launch_tma_mode_##ST<1>(A, maps, tma_ok, single, s);                           \
            case 2: return launch_tma_mode_##ST<2>(A, maps, tma_ok, single, s);                           \
            case 3: return launch_tma_mode_##ST<3>(A, maps, tma_ok, single, s);                           \
            case 4: return launch_tma_mode_##ST<4>(A, maps, tma_ok, single, s);                           \
        }                                                                                                 \
        return cudaErrorInvalidValue;                                                                     \
    }                                                                                                     \
    template <>                                                                                           \
    bool tma_supported<ST>(int nc) {                                                                      \
        switch (nc) {                                                                                     \
            case 1: return TmaLayout<1, ST, kTmaTileY>::fits;                                             \
            case 2: return TmaLayout<2, ST, kTmaTileY>::fits;                                             \
            case 3: return TmaLayout<3, ST, kTmaTileY>::fits;                                             \
            case 4: return TmaLayout<4, ST, kTmaTileY>::fits;                                             \
        }                                                                                                 \
        return false;                                                                                     \
    }


#define FMLBM_DEFINE_MULTI_LAUNCHER(ST)                                                                   \
    template <int NC>                                                                                     \
    static cudaError_t launch_multi_nc_##ST(const StepArgs& A0, const StepArgs& A1, int nsteps,           \
                                            long long* done, cudaStream_t s) {                            \
        constexpr int TY = kTileYSmall;                                                                   \
        constexpr size_t smem = sizeof(StepSmem<float, NC, TY>) + park_bytes<NC, ST, TY>();               \
        auto k = fused_steps<NC, ST, TY>;                                                                 \
        FMLBM_ENSURE_SMEM(k, smem);                                                                       \
        int dev = 0, sms = 0, per_sm = 0;                                                                 \
        cudaError_t e = cudaGetDevice(&dev);                                                              \
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);      \
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kTX * TY, smem); \
        if (e != cudaSuccess) return e;                                                                   \
        if (per_sm < 1) return cudaErrorInvalidConfiguration;                                             \
        const int ntiles = multi_tiles(A0.nx, A0.ny);                                                     \
        const int grid = ntiles < sms * per_sm ? ntiles : sms * per_sm;                                   \
        e = cudaMemsetAsync(done, 0, (size_t)ntiles * sizeof(long long), s);                              \
        if (e != cudaSuccess) return e;                                                                   \
        Planes P0 = make_planes(A0, NC, ST != ST_F32, ST == ST_F32 ? 4 : 2);                              \
        Planes P1 = make_planes(A1, NC, ST != ST_F32, ST == ST_F32 ? 4 : 2);                              \
        StepArgs a0 = A0, a1 = A1;                                                                        \
        long long base = 0;                                                                               \
        void* args[] = {&a0, &a1, &P0, &P1, &nsteps, &base, &done};                                       \
        return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k), dim3(grid), dim3(kTX, TY), args, smem, s); \
    }                                                                                                     \
    template <>                                                                                           \
    cudaError_t launch_steps_multi<ST>(const StepArgs& A0, const StepArgs& A1, int nc, int nsteps,        \
                                       long long* done, cudaStream_t s) {                                 \
        if (!spec_options(A0)) return cudaErrorNotSupported;                                              \
        switch (nc) {                                                                                     \
            case 1: return launch_multi_nc_##ST<1>(A0, A1, nsteps, done, s);                             \
            case 2: return launch_multi_nc_##ST<2>(A0, A1, nsteps, done, s);                              \
            case 3: return launch_multi_nc_##ST<3>(A0, A1, nsteps, done, s);                              \
            case 4: return launch_multi_nc_##ST<4>(A0, A1, nsteps, done, s);                              \
        }                                                                                                 \
        return cudaErrorInvalidValue;                                                                     \
    }

// Components parked in shared memory by the paired step: registers hold the others'
// pulled values of both nodes between phases 1 and 3.
template <int NC> constexpr int kPairPark = NC == 1 ? 0 : (NC == 2 ? 1 : 2);

#define FMLBM_DEFINE_PAIR_LAUNCHER(ST)                                                                    \
    template <int NC, bool LAG>                                                                           \
    static cudaError_t launch_pair_lag_##ST(const StepArgs& A, cudaStream_t s) {                          \
        constexpr int NP = kPairPark<NC>;                                                                 \
        constexpr size_t smem = pair_smem_bytes<NC, ST, kTileYSmall, NP>();                                   \
        auto k = fused_step_pair<NC, ST, kTileYSmall, NP, LAG>;                                           \
        FMLBM_ENSURE_SMEM(k, smem);                                                                       \
        dim3 grid((A.nx + kPW - 1) / kPW, (A.ny + kTileYSmall - 1) / kTileYSmall);                        \
        const Planes P = make_planes(A, NC, ST == ST_F16DEV || ST == ST_BF16DEV, ST == ST_F32 ? 4 : 2);   \
        k<<<grid, dim3(kTX, kTileYSmall), smem, s>>>(A, P);                                               \
        return cudaGetLastError();                                                                        \
    }                                                                                                     \
    template <int NC>                                                                                     \
    static cudaError_t launch_pair_nc_##ST(const StepArgs& A, cudaStream_t s) {                           \
        return A.lagged ? launch_pair_lag_##ST<NC, true>(A, s) : launch_pair_lag_##ST<NC, false>(A, s);   \
    }                                                                                                     \
    template <>                                                                                           \
    cudaError_t launch_step_pair<ST>(const StepArgs& A, int nc, cudaStream_t s) {                         \
        switch (nc) {                                                                                     \
            case 1: return launch_pair_nc_##ST<1>(A, s);                                                  \
            case 2: return launch_pair_nc_##ST<2>(A, s);                                                  \
            case 3: return launch_pair_nc_##ST<3>(A, s);                                                  \
            case 4: return launch_pair_nc_##ST<4>(A, s);                                                  \
        }                                                                                                 \
        return cudaErrorInvalidValue;                                                                     \
    }                                                                                                     \
    template <>                                                                                           \
    bool pair_supported<ST>(int nc) {                                                                     \
        return nc >= 1 && nc <= 4;                                                                        \
    }

}  // namespace fmlbm
