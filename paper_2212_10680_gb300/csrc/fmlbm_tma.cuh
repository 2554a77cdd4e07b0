// TMA-fed persistent variant of the fused step (sm_103a, float and 16-bit storage).
//
// Each block stays resident and walks a strided list of 32 x TY tiles.  For a tile that
// needs no periodic wrap, one elected thread issues a single 3-D bulk tensor copy
// (cp.async.bulk.tensor) of every distribution plane of the tile plus its 3-node pull
// halo into shared memory, completing on an mbarrier; with two stages the copy of the
// next tile is in flight while the current one is computed.  Tiles on the periodic
// edges take the plain pull path of fused_step.  Both paths run the same phase
// functions, so the results are bit-identical to fused_step.
//
// Box of one stage: columns x0 - 4 .. x0 + 35 (x0 - 8 .. x0 + 39 for 16-bit planes, so
// that the innermost coordinate times the element size is a multiple of 16 bytes), rows
// y0 - 3 .. y0 + TY + 2, all planes.  Every wait on an mbarrier is bounded (A.wait_polls
// polls for a tile's copy); a wait that runs out latches error code 2 and the block waits
// (bounded, at the full limit) for its copies in flight and returns.
#pragma once

#include <cuda.h>

#include "fmlbm_kernels.cuh"

namespace fmlbm {

constexpr int kTmaTileY = 8;
constexpr long long kMaxPolls = 1ll << 24;  // try_wait polls before a wait is declared failed

template <int ST> struct TmaGeom;
template <> struct TmaGeom<ST_F32> {
    static constexpr int W = kTX + 8;        // float planes, origin x0 - 4
    static constexpr int W16 = 0;
};
template <> struct TmaGeom<ST_F16DEV> {
    static constexpr int W = kTX + 8;        // float a = 0 planes, origin x0 - 4
    static constexpr int W16 = kTX + 16;     // 16-bit planes, origin x0 - 8
};
template <> struct TmaGeom<ST_BF16DEV> : TmaGeom<ST_F16DEV> {};

template <int NC, int ST, int TY>
struct TmaLayout {
    static constexpr int H = TY + 6;
    static constexpr int W = TmaGeom<ST>::W;
    static constexpr int W16 = TmaGeom<ST>::W16;
    static constexpr bool dev = ST != ST_F32;
    static constexpr size_t f32_planes = dev ? NC : 9 * NC;
    static constexpr size_t f32_bytes = f32_planes * H * W * 4;
    static constexpr size_t b16_bytes = dev ? (size_t)8 * NC * H * W16 * 2 : 0;
    static constexpr size_t align128(size_t v) { return (v + 127) & ~size_t(127); }
    static constexpr size_t stage_bytes = align128(f32_bytes) + align128(b16_bytes);
    // the step's shared tiles, then the diagnostics snapshot copy of the tile's nodes
    static constexpr size_t scratch_bytes = align128(sizeof(StepSmem<float, NC, TY>) + (size_t)NC * TY * kTX * 4);
    static constexpr int stages = (scratch_bytes + 2 * stage_bytes + 64 <= 220 * 1024) ? 2 : 1;
    static constexpr size_t smem_bytes = scratch_bytes + stages * stage_bytes + 64;
    static constexpr bool fits = smem_bytes <= 227 * 1024;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: true once the phase with this parity has completed, false after `polls`
// polls (none at all for polls <= 0).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long polls = kMaxPolls) {
    for (long long k = 0; k < polls; ++k)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// Pulled value of plane (i, a) for box position (col, row) of the x0 - 4 origin.
template <int NC, int ST, int TY>
__device__ __forceinline__ typename StoreTraits<ST>::Real stage_value(const unsigned char* stage, int i, int a,
                                                                      int row, int col) {
    using L = TmaLayout<NC, ST, TY>;
    const float* f = reinterpret_cast<const float*>(stage);
    if constexpr (ST == ST_F32) {
        return f[((i * 9 + a) * L::H + row) * L::W + col];
    } else {
        using Elem = typename StoreTraits<ST>::Elem;
        if (a == 0) return f[(i * L::H + row) * L::W + col];
        const Elem* h = reinterpret_cast<const Elem*>(stage + L::align128(L::f32_bytes));
        return to_real(h[((i * 8 + a - 1) * L::H + row) * L::W16 + col + 4]);
    }
}

// NSTAGE = 2: persistent blocks, the next tile's copy overlaps this tile's arithmetic; each
// thread keeps its node's pulled values in registers between the phases.
// NSTAGE = 1: one tile per block (grid = tile count), MINB blocks resident per SM; the
// pulled values stay in shared memory between the phases (the stage for copied tiles, the
// same bytes as a compact [9N][TY][32] array for edge tiles), which keeps the register
// count within MINB blocks per SM.
template <int NC, int ST, int TY, int NSTAGE, int MINB>
__global__ void __launch_bounds__(kTX* TY, MINB)
    fused_step_tma(const __grid_constant__ StepArgs A, const __grid_constant__ CUtensorMap map_f32,
                   const __grid_constant__ CUtensorMap map_b16, int tma_ok) {
    using Real = typename StoreTraits<ST>::Real;
    using L = TmaLayout<NC, ST, TY>;
    static_assert((size_t)9 * NC * TY * kTX * sizeof(Real) <= L::stage_bytes, "edge tiles park g in the stage");
    extern __shared__ __align__(128) unsigned char smem_tma[];
    auto& S = *reinterpret_cast<StepSmem<Real, NC, TY>*>(smem_tma);
    unsigned char* stages = smem_tma + L::scratch_bytes;
    Real* pv_s = reinterpret_cast<Real*>(smem_tma + sizeof(StepSmem<Real, NC, TY>));
    uint64_t* bar = reinterpret_cast<uint64_t*>(stages + NSTAGE * L::stage_bytes);
    const MixConstT<Real>& m = mixc<Real>(A);

    const int nx = A.nx, ny = A.ny;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * kTX + tx;
    const int tiles_x = (nx + kTX - 1) / kTX;
    const int ntiles = tiles_x * ((ny + TY - 1) / TY);

    auto origin = [&](int t, int& x0, int& y0) {
        x0 = (t % tiles_x) * kTX;
        y0 = (t / tiles_x) * TY;
    };
    auto is_inner = [&](int x0, int y0) { return x0 >= 3 && x0 + kTX + 3 <= nx && y0 >= 3 && y0 + TY + 3 <= ny; };
    auto use_tma = [&](int t) {
        int x0, y0;
        origin(t, x0, y0);
        return tma_ok && is_inner(x0, y0);
    };
    auto issue = [&](int t, int s) {  // one elected thread
        int x0, y0;
        origin(t, x0, y0);
        unsigned char* st = stages + s * L::stage_bytes;
        mbar_expect_tx(&bar[s], (uint32_t)(L::f32_bytes + L::b16_bytes));
        tma_load_3d(st, &map_f32, &bar[s], x0 - 4, y0 - 3, 0);
        if constexpr (L::dev) tma_load_3d(st + L::align128(L::f32_bytes), &map_b16, &bar[s], x0 - 8, y0 - 3, 0);
    };

    if (tid == 0) {
        for (int s = 0; s < NSTAGE; ++s) mbar_init(&bar[s]);
        mbar_fence_init();
    }
    __syncthreads();

    uint32_t parity = 0u;   // bit s: phase parity the next wait on stage s expects
    uint32_t pending = 0u;  // bit s: a copy into stage s is in flight
    int t = blockIdx.x;
    if (NSTAGE == 2 && t < ntiles && use_tma(t)) {
        if (tid == 0) issue(t, 0);
        pending |= 1u;
    }
    for (int k = 0; t < ntiles; t += gridDim.x, ++k) {
        const int s = NSTAGE == 2 ? (k & 1) : 0;
        const bool tma_here = use_tma(t);
        if (NSTAGE == 2) {
            const int tn = t + gridDim.x;
            if (tn < ntiles && use_tma(tn)) {
                if (tid == 0) issue(tn, s ^ 1);
                pending |= 1u << (s ^ 1);
            }
        } else if (tma_here) {
            if (tid == 0) issue(t, 0);
            pending |= 1u;
        }
        int x0, y0;
        origin(t, x0, y0);
        const int gxn = x0 + tx, gyn = y0 + ty;
        prefetch_force<Real, NC, TY>(A, S, tx, ty, gxn, gyn);
        diag_prefetch<NC, Real, TY>(A, pv_s, tx, ty, gxn, gyn);
        unsigned char* st = stages + s * L::stage_bytes;
        Real* gpark = reinterpret_cast<Real*>(st);  // edge tiles: [9N][TY][32]
        constexpr bool PARK = NSTAGE == 1;
        Real g[NC][9], r[NC], jx, jy;
        if (tma_here) {
            const bool ok = mbar_wait_bounded(&bar[s], (parity >> s) & 1u, A.wait_polls);
            if (__syncthreads_or(!ok)) {
                // a wait ran out: report, wait (at the full limit) for every copy still in
                // flight into this block's shared memory, the one waited for included, so that
                // none lands after the block has gone, and leave
                if (tid == 0 && atomicCAS(&A.err->flag, 0, 2) == 0) {
                    A.err->comp = -1;
                    A.err->x = x0;
                    A.err->y = y0;
                }
#pragma unroll
                for (int q = 0; q < NSTAGE; ++q)
                    if ((pending >> q) & 1u) mbar_wait_bounded(&bar[q], (parity >> q) & 1u);
                asm volatile("cp.async.wait_all;\n" ::: "memory");  // the force prefetch
                return;
            }
            parity ^= 1u << s;
            pending &= ~(1u << s);
#pragma unroll
            for (int a = 0; a < 9; ++a)
#pragma unroll
                for (int i = 0; i < NC; ++i)
                    g[i][a] = stage_value<NC, ST, TY>(st, i, a, ty + 3 - ey(a), tx + 4 - ex(a));
            phase1_node<NC, TY, Real>(A, m, S, g, r, jx, jy, tx, ty, gxn < nx && gyn < ny, gxn, gyn);
            constexpr int RING = 4 * (kTX + 4) + 4 * TY;
            for (int r = tid; r < RING; r += kTX * TY) {
                int bx, by;
                ring_position<TY>(r, bx, by);
                Real rt[NC];
#pragma unroll
                for (int a = 0; a < 9; ++a)
#pragma unroll
                    for (int i = 0; i < NC; ++i) {
                        const Real v = stage_value<NC, ST, TY>(st, i, a, by + 1 - ey(a), bx + 2 - ex(a));
                        rt[i] = a == 0 ? v : vadd(rt[i], v);  // the order of pull_rho
                    }
                phase1_ring<NC, TY, Real>(A, m, S, rt, bx, by);
            }
        } else {
            phase1_global<NC, ST, TY>(A, m, S, g, r, jx, jy, x0, y0, is_inner(x0, y0), tx, ty, tid);
            if constexpr (PARK) {
#pragma unroll
                for (int i = 0; i < NC; ++i)
#pragma unroll
                    for (int a = 0; a < 9; ++a) gpark[((i * 9 + a) * TY + ty) * kTX + tx] = g[i][a];
            }
        }
        __syncthreads();
        phase2<NC, TY, Real>(m, S, A.stencil, tid);
        __syncthreads();
        if (gxn < nx && gyn < ny) {
            if constexpr (PARK) {
#pragma unroll
                for (int a = 0; a < 9; ++a)
#pragma unroll
                    for (int i = 0; i < NC; ++i)
                        g[i][a] = tma_here ? stage_value<NC, ST, TY>(st, i, a, ty + 3 - ey(a), tx + 4 - ex(a))
                                           : gpark[((i * 9 + a) * TY + ty) * kTX + tx];
            }
            phase3<NC, ST, TY, false>(A, m, S, g, r, jx, jy, tx, ty, gxn, gyn);
        }
        if (A.diag_partial != nullptr)  // uniform: diagnostics of the state this step read
            diag_tile<NC, Real, TY>(A, r, pv_s, tx, ty, gxn, gyn, y0, t / tiles_x, t % tiles_x, tiles_x);
        __syncthreads();  // shared tiles and the stage are free again
    }
}

}  // namespace fmlbm
