// Multi-step persistent variant of the specialised fused step (sm_103a, float and 16-bit
// storage; Peng-Robinson EOS, isotropic stencils, lagged velocity, well-balanced scheme).
//
// One cooperative launch advances a lattice by K time steps.  Its blocks are all resident;
// each walks a fixed list of 32 x TY tiles once per step.  A tile's update at step s reads
// distributions up to three nodes away (the pulls of its 2-node halo ring), so it depends
// only on the 3 x 3 neighbourhood of tiles (tiles are at least 8 x 32 nodes): it may start
// once those nine tiles have completed step s - 1.  That also covers the write-after-read
// hazard: step s writes the buffer step s - 1 read, and those reads were the neighbours'.
// Every tile publishes the number of steps it has completed in done[tile] (a release store
// after the block's stores; readers poll with acquire loads, bounded by A.wait_polls polls,
// after which the block latches error 2 and leaves; the blocks waiting on it then run out of
// polls too, so the launch always ends).  Neighbours are therefore never more than one step
// apart, and no block waits on a step later than its own, so with all blocks resident every
// wait ends.
//
// Steps overlap: a block that has finished its tiles of step s goes on with step s + 1 wherever
// the neighbourhood is ready, so the per-launch ramp (every block waiting for its first loads)
// and tail (a few blocks finishing) of single-step launches occur once per K steps, and a step
// reads much of what the previous step wrote while it is still in L2.  Tiles are visited in
// row order folded from both ends (rows 0, R-1, 1, R-2, ...), so that the periodic neighbours
// of the first and last rows are visited at the same point of every step.
//
// The distributions are read through L2 only (ld.global.cg: other multiprocessors write them
// during the launch); the stored force and the tiles' own values are read and written by the
// same block.  The arithmetic per tile is that of fused_step, so the results are bit-identical
// to K single steps.
#pragma once

#include "fmlbm_kernels.cuh"

namespace fmlbm {

__device__ __forceinline__ long long ld_acquire_gpu(const long long* p) {
    long long v;
    asm volatile("ld.acquire.gpu.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(long long* p, long long v) {
    asm volatile("st.release.gpu.global.s64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// The q-th tile of the visiting order: rows folded from both ends, columns in order.
__device__ __forceinline__ void folded_tile(int q, int tiles_x, int tiles_y, int& tcx, int& tcy) {
    const int k = q / tiles_x;
    tcx = q - k * tiles_x;
    tcy = (k & 1) ? tiles_y - 1 - (k >> 1) : (k >> 1);
}

// One tile's update: the body of the specialised fused_step with the tile origin given.
template <int NC, int ST, int TY>
__device__ __forceinline__ void multi_tile(const StepArgs& A, const Planes& P, unsigned char* smem_raw, int tcx,
                                           int tcy, int tiles_x) {
    using Real = typename StoreTraits<ST>::Real;
    constexpr bool PARK = kParkLast<NC, ST, TY>;
    auto& S = *reinterpret_cast<StepSmem<Real, NC, TY>*>(smem_raw);
    Real* park = reinterpret_cast<Real*>(smem_raw + sizeof(StepSmem<Real, NC, TY>));
    const MixConstT<Real>& m = mixc<Real>(A);
    const int nx = A.nx, ny = A.ny;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * kTX + tx;
    const int x0 = tcx * kTX, y0 = tcy * TY;
    const bool inner = x0 >= 3 && x0 + kTX + 3 <= nx && y0 >= 3 && y0 + TY + 3 <= ny;
    const int gxn = x0 + tx, gyn = y0 + ty;
    prefetch_force<Real, NC, TY>(A, S, tx, ty, gxn, gyn, 1);
    Real g[NC][9], r[NC], jx, jy;
    if (inner)
        phase1_global<NC, ST, TY, PARK, 1, true>(A, m, S, g, r, jx, jy, x0, y0, true, tx, ty, tid, &P, 0);
    else
        phase1_global<NC, ST, TY, PARK, 0, true>(A, m, S, g, r, jx, jy, x0, y0, false, tx, ty, tid, &P, 0);
    if constexpr (PARK) park_store<TY, Real>(g[NC - 1], park, tid);
    __syncthreads();
    phase2<NC, TY, Real>(m, S, 0, tid);
    __syncthreads();
    if (gxn < nx && gyn < ny)
        phase3<NC, ST, TY, false, false, PARK, PARK>(A, m, S, g, r, jx, jy, tx, ty, gxn, gyn, park, &P, 0, 1);
    (void)tiles_x;
}

// A0 / P0: the arguments of the launch's even steps (reading the current buffer), A1 / P1 of
// its odd steps.  done: ntiles counters, all equal to base when the launch starts.
// Registers: the loop state and the two parameter sets cost registers over fused_step, which
// at the same occupancy spills; 64 registers (four blocks per SM) for up to two components,
// 80 (three blocks) for more, the fastest measured forms without spills.
template <int NC, int ST, int TY>
__global__ void __launch_bounds__(kTX* TY, NC <= 2 ? 4 : 3)
    fused_steps(const __grid_constant__ StepArgs A0, const __grid_constant__ StepArgs A1,
                const __grid_constant__ Planes P0, const __grid_constant__ Planes P1, int nsteps, long long base,
                long long* __restrict__ done) {
    static_assert(ST == ST_F32 || ST == ST_F16DEV || ST == ST_BF16DEV, "float and 16-bit storage");
    extern __shared__ __align__(16) unsigned char smem_multi[];
    const int tid = threadIdx.y * kTX + threadIdx.x;
    const int tiles_x = (A0.nx + kTX - 1) / kTX, tiles_y = (A0.ny + TY - 1) / TY;
    const int ntiles = tiles_x * tiles_y;
    for (int s = 0; s < nsteps; ++s) {
        for (int q = blockIdx.x; q < ntiles; q += gridDim.x) {
            int tcx, tcy;
            folded_tile(q, tiles_x, tiles_y, tcx, tcy);
            bool late = false;
            if (s > 0 && tid < 9) {  // the 3 x 3 neighbourhood has completed step s - 1
                const int ux = wrap(tcx + tid % 3 - 1, tiles_x), uy = wrap(tcy + tid / 3 - 1, tiles_y);
                const long long* f = done + (size_t)uy * tiles_x + ux;
                long long polls = 0;
                while (ld_acquire_gpu(f) < base + s) {
                    if (++polls > A0.wait_polls) {
                        late = true;
                        break;
                    }
                    __nanosleep(64);
                }
            }
            if (__syncthreads_or(late)) {
                if (tid == 0 && atomicCAS(&A0.err->flag, 0, 2) == 0) {
                    A0.err->comp = -1;
                    A0.err->x = tcx * kTX;
                    A0.err->y = tcy * TY;
                }
                asm volatile("cp.async.wait_all;\n" ::: "memory");
                return;
            }
            // the step's arguments as compile-time references to the launch parameters (a runtime
            // choice between them turns every constant operand into a load)
            if ((s & 1) == 0)
                multi_tile<NC, ST, TY>(A0, P0, smem_multi, tcx, tcy, tiles_x);
            else
                multi_tile<NC, ST, TY>(A1, P1, smem_multi, tcx, tcy, tiles_x);
            __syncthreads();  // the tile's stores are issued and its shared tiles free again
            if (tid == 0) {
                __threadfence();
                st_release_gpu(done + (size_t)tcy * tiles_x + tcx, base + s + 1);
            }
        }
    }
}

}  // namespace fmlbm
