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

// Per-item partial sums (2 NC + 2 doubles: sum rho_i, sum (rho - rho_prev)^2, sum rho^2, then
// the phase measure's sum ln rho_i) over the item's tile of 32 x tile_y nodes, then
// rho_prev <- rho, with the node sums, the warp tree and the double strip sums of
// reduce_partial and lnrho_partial (the rows of a taller tile go through the same
// compensated sums before the tree).  The items of one lattice are contiguous, so
// batch_reduce_final sums each lattice in a fixed order.
template <int NC>
constexpr int kBatchSums = 2 * NC + 2;

template <int NC, int ST>
__global__ void __launch_bounds__(kTX* 8) batch_reduce(BatchLattice* __restrict__ lat, const WorkItem* __restrict__ work,
                                                       int nwork, void* const* __restrict__ rho_prev,
                                                       double* __restrict__ partial) {
    using Real = typename StoreTraits<ST>::Real;
    constexpr int K = kBatchSums<NC>;
    const int w = blockIdx.x;
    if (w >= nwork) return;
    const WorkItem it = work[w];
    const BatchLattice* L = lat + it.lattice;
    const StepArgs& A = L->args[L->step & 1];
    const int nx = A.nx, ny = A.ny, nxy = nx * ny;
    Real* prev = static_cast<Real*>(rho_prev[it.lattice]);
    Sum2<Real> acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = s2_of(Real(0));
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
                Sum2<Real> a[NC + 2], l[NC];
                diag_node<NC, Real>(r, pv, 1, a);
                lnrho_node<NC, Real>(r, l);
#pragma unroll
                for (int k = 0; k < NC + 2; ++k) acc[k] = s2_add(acc[k], a[k]);
#pragma unroll
                for (int i = 0; i < NC; ++i) acc[NC + 2 + i] = s2_add(acc[NC + 2 + i], l[i]);
#pragma unroll
                for (int i = 0; i < NC; ++i) prev[(size_t)i * nxy + node] = r[i];
            }
        }
    }
    __shared__ Sum2<Real> red[8][K];
    sums_warp<K, Real>(acc, red[threadIdx.y]);
    __syncthreads();
    const int tid = threadIdx.y * kTX + threadIdx.x;
    if (tid < K) partial[(size_t)w * K + tid] = sums_strip<K, Real>(red, 0, tid, 0);
}

template <int NC>
__global__ void batch_reduce_final(const BatchLattice* __restrict__ lat, int n, const double* __restrict__ partial,
                                   double* __restrict__ out) {
    constexpr int K = kBatchSums<NC>;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n * K) return;
    const int l = k / K, q = k % K;
    double v = 0.0;
    for (int w = lat[l].item0; w < lat[l].item0 + lat[l].nitems; ++w) v += partial[(size_t)w * K + q];
    out[k] = v;
}

// The two phases of a lattice from its densities rho[N][ny][nx] (mass, double), read as
// means over 2 x 2 blocks of nodes (block (bx, by) holds the nodes 2 bx, 2 bx + 1 in x and
// 2 by, 2 by + 1 in y, periodic at an odd edge).  The discrete force of Eqs. eqforcefinal and
// eq1stder differences a field over two nodes, so a field alternating from node to node (a
// checkerboard) feels no force, and at rest the well-balanced equilibrium (rho_0 = 0) holds
// every node's mass in its rest population, so nothing streams it away either: a checkerboard
// that the transient of a sharp interface excites stays in both bulk phases.  Each parity
// sublattice is then out of equilibrium on its own; the block mean is the thermodynamic state.
// out = the block-mean molar densities rho~_i at the block of largest total molar density
// sum_i rho_i / M_i (liquid) [N], then at the block of smallest (vapour) [N]; ties to the
// lowest block index (row-major).  One block of threads, grid-stride over the node blocks, a
// fixed-order tree: deterministic.
constexpr int kPhaseThreads = 512;
__device__ __forceinline__ void block_nodes(long long k, int nx, int ny, long long (&node)[4]) {
    const int bxn = (nx + 1) / 2;
    const int x0 = 2 * (int)(k % bxn), y0 = 2 * (int)(k / bxn);
    const int x1 = x0 + 1 < nx ? x0 + 1 : 0, y1 = y0 + 1 < ny ? y0 + 1 : 0;
    node[0] = (long long)y0 * nx + x0;
    node[1] = (long long)y0 * nx + x1;
    node[2] = (long long)y1 * nx + x0;
    node[3] = (long long)y1 * nx + x1;
}

template <int NC>
__global__ void __launch_bounds__(kPhaseThreads) phase_nodes(const double* __restrict__ rho, int nx, int ny,
                                                             MixConstT<double> m, double* __restrict__ out) {
    __shared__ double vmax[kPhaseThreads], vmin[kPhaseThreads];
    __shared__ long long imax[kPhaseThreads], imin[kPhaseThreads];
    const long long nxy = (long long)nx * ny;
    const long long nblk = (long long)((nx + 1) / 2) * ((ny + 1) / 2);
    const int t = threadIdx.x;
    double hi = -1.0, lo = 0.0;
    long long ih = -1, il = -1;
    for (long long k = t; k < nblk; k += kPhaseThreads) {
        long long node[4];
        block_nodes(k, nx, ny, node);
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int i = 0; i < NC; ++i) s += rho[i * nxy + node[q]] / m.M[i];
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
    if (t < 2 * NC) {
        const int i = t % NC;
        long long node[4];
        block_nodes(t < NC ? imax[0] : imin[0], nx, ny, node);
        double v = 0.0;
#pragma unroll
        for (int q = 0; q < 4; ++q) v += rho[i * nxy + node[q]] / m.M[i];
        out[t] = 0.25 * v;
    }
}

}  // namespace fmlbm
