// Batched lattices: many independent lattices (same component count and storage,
// any sizes, any mixtures) advanced together by one persistent kernel per time step.
//
// Every lattice has a device-resident descriptor holding its StepArgs for both
// step parities (the ping-pong buffers swapped) and its own step counter.  A work list
// of (lattice, tile) items covers all lattices; a block copies the descriptor of its
// item's lattice into shared memory and runs the same phase functions as fused_step,
// so each lattice's arithmetic is exactly that of a single-lattice plain step: results
// are bit-identical alone and in any mix.  Retired lattices are skipped through a
// device flag, so a captured graph of the step loop stays valid as lattices retire.
#pragma once

#include "fmlbm_kernels.cuh"

namespace fmlbm {

struct BatchLattice {
    StepArgs args[2];    // [step & 1]
    long long step;      // steps taken (device side, advanced by batch_advance)
    int active;          // 0: retired or not started
    int item0, nitems;   // its items in the work list
    int tile_y;          // the tile height its items were cut with
    int pad[3];
};

struct WorkItem {
    int lattice;
    int x0, y0;
};

// One step of every active lattice.
// Float storage capped at 64 registers (1024 threads per SM), as the single-lattice step.
template <int NC, int ST, int TY>
__global__ void __launch_bounds__(kTX* TY, ST == ST_F64 ? 1 : 1024 / (kTX * TY)) batch_step(BatchLattice* __restrict__ lat,
                                                      const WorkItem* __restrict__ work, int nwork) {
    using Real = typename StoreTraits<ST>::Real;
    extern __shared__ __align__(16) unsigned char smem_batch[];
    auto& S = *reinterpret_cast<StepSmem<Real, NC, TY>*>(smem_batch);
    __shared__ __align__(16) StepArgs As;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * kTX + tx;
    constexpr int NT = kTX * TY;
    constexpr int WORDS = sizeof(StepArgs) / 4;
    static_assert(sizeof(StepArgs) % 4 == 0, "StepArgs copied as words");
    for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
        const WorkItem it = work[w];
        const BatchLattice* L = lat + it.lattice;
        if (!L->active) continue;  // uniform across the block
        const int* src = reinterpret_cast<const int*>(&L->args[L->step & 1]);
        int* dst = reinterpret_cast<int*>(&As);
        for (int k = tid; k < WORDS; k += NT) dst[k] = src[k];
        __syncthreads();
        const StepArgs& A = As;
        const MixConstT<Real>& m = mixc<Real>(A);
        const int nx = A.nx, ny = A.ny;
        const int x0 = it.x0, y0 = it.y0;
        const bool inner = x0 >= 3 && x0 + kTX + 3 <= nx && y0 >= 3 && y0 + TY + 3 <= ny;
        const int gxn = x0 + tx, gyn = y0 + ty;
        prefetch_force<Real, NC, TY>(A, S, tx, ty, gxn, gyn);
        Real g[NC][9], r[NC], jx, jy;
        phase1_global<NC, ST, TY>(A, m, S, g, r, jx, jy, x0, y0, inner, tx, ty, tid);
        __syncthreads();
        phase2<NC, TY, Real>(m, S, A.stencil, tid);
        __syncthreads();
        if (gxn < nx && gyn < ny) phase3<NC, ST, TY, false>(A, m, S, g, r, jx, jy, tx, ty, gxn, gyn);
        __syncthreads();  // As and the shared tiles are reused by the next item
    }
}

__global__ void batch_advance(BatchLattice* __restrict__ lat, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n && lat[k].active) lat[k].step += 1;
}

// Per-item partial sums (NC + 2 doubles: sum rho_i, sum (rho - rho_prev)^2, sum rho^2) over
// the item's tile of 32 x tile_y nodes, then rho_prev <- rho, with the node sums, the warp
// tree and the double strip sums of reduce_partial (the rows of a taller tile go through the
// same compensated sums before the tree).  The items of one lattice are contiguous, so
// batch_reduce_final sums each lattice in a fixed order.
template <int NC, int ST>
__global__ void __launch_bounds__(kTX* 8) batch_reduce(BatchLattice* __restrict__ lat, const WorkItem* __restrict__ work,
                                                       int nwork, void* const* __restrict__ rho_prev,
                                                       double* __restrict__ partial) {
    using Real = typename StoreTraits<ST>::Real;
    const int w = blockIdx.x;
    if (w >= nwork) return;
    const WorkItem it = work[w];
    const BatchLattice* L = lat + it.lattice;
    const StepArgs& A = L->args[L->step & 1];
    const int nx = A.nx, ny = A.ny, nxy = nx * ny;
    Real* prev = static_cast<Real*>(rho_prev[it.lattice]);
    Sum2<Real> acc[NC + 2];
#pragma unroll
    for (int k = 0; k < NC + 2; ++k) acc[k] = s2_of(Real(0));
    if (L->active) {
        for (int ry = threadIdx.y; ry < L->tile_y; ry += 8) {
            const int x = it.x0 + threadIdx.x, y = it.y0 + ry;
            if (x < nx && y < ny) {
                const bool inner = x >= 1 && x + 1 < nx && y >= 1 && y + 1 < ny;
                Real r[NC];
                pull_rho<NC, ST>(A, x, y, inner, nx, ny, nxy, r);
                const int node = y * nx + x;
                Real pv[NC];
#pragma unroll
                for (int i = 0; i < NC; ++i) pv[i] = prev[(size_t)i * nxy + node];
                Sum2<Real> a[NC + 2];
                diag_node<NC, Real>(r, pv, 1, a);
#pragma unroll
                for (int k = 0; k < NC + 2; ++k) acc[k] = s2_add(acc[k], a[k]);
#pragma unroll
                for (int i = 0; i < NC; ++i) prev[(size_t)i * nxy + node] = r[i];
            }
        }
    }
    __shared__ Sum2<Real> red[8][NC + 2];
    diag_warp<NC, Real>(acc, red[threadIdx.y]);
    __syncthreads();
    const int tid = threadIdx.y * kTX + threadIdx.x;
    if (tid < NC + 2) partial[(size_t)w * (NC + 2) + tid] = diag_strip<NC, Real>(red, 0, tid, 0);
}

template <int NC>
__global__ void batch_reduce_final(const BatchLattice* __restrict__ lat, int n, const double* __restrict__ partial,
                                   double* __restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n * (NC + 2)) return;
    const int l = k / (NC + 2), q = k % (NC + 2);
    double v = 0.0;
    for (int w = lat[l].item0; w < lat[l].item0 + lat[l].nitems; ++w) v += partial[(size_t)w * (NC + 2) + q];
    out[k] = v;
}

// The two phases of a lattice from its densities rho[N][nxy] (mass, double): the node of
// largest total molar density sum_i rho_i / M_i (liquid) and of smallest (vapour), ties to
// the lowest node index; out = rho~ at the liquid node [N], then at the vapour node [N].
// One block, grid-stride over the nodes, a fixed-order tree: deterministic.
constexpr int kPhaseThreads = 512;
template <int NC>
__global__ void __launch_bounds__(kPhaseThreads) phase_nodes(const double* __restrict__ rho, long long nxy,
                                                             MixConstT<double> m, double* __restrict__ out) {
    __shared__ double vmax[kPhaseThreads], vmin[kPhaseThreads];
    __shared__ long long imax[kPhaseThreads], imin[kPhaseThreads];
    const int t = threadIdx.x;
    double hi = -1.0, lo = 0.0;
    long long ih = -1, il = -1;
    for (long long k = t; k < nxy; k += kPhaseThreads) {
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < NC; ++i) s += rho[i * nxy + k] / m.M[i];
        if (ih < 0 || s > hi) { hi = s; ih = k; }          // k increases: first maximum kept
        if (il < 0 || s < lo) { lo = s; il = k; }
    }
    vmax[t] = hi; imax[t] = ih; vmin[t] = lo; imin[t] = il;
    __syncthreads();
    for (int w = kPhaseThreads / 2; w > 0; w >>= 1) {
        if (t < w) {
            const int o = t + w;
            if (imax[o] >= 0 && (imax[t] < 0 || vmax[o] > vmax[t] || (vmax[o] == vmax[t] && imax[o] < imax[t]))) {
                vmax[t] = vmax[o]; imax[t] = imax[o];
            }
            if (imin[o] >= 0 && (imin[t] < 0 || vmin[o] < vmin[t] || (vmin[o] == vmin[t] && imin[o] < imin[t]))) {
                vmin[t] = vmin[o]; imin[t] = imin[o];
            }
        }
        __syncthreads();
    }
    if (t < NC) {
        out[t] = rho[t * nxy + imax[0]] / m.M[t];
        out[NC + t] = rho[t * nxy + imin[0]] / m.M[t];
    }
}

}  // namespace fmlbm
