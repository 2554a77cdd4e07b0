// The paired step kernel (sm_103a, float and 16-bit storage): one time step of the method
// (Section III.B, steps 1-9), each thread advancing two nodes of a 64 x TY tile, 32
// columns apart.
//
// The per-node arithmetic is the lane arithmetic of fmlbm_kernels.cuh with two lanes
// (float2): every float operation of the two nodes issues as one packed f32x2 instruction,
// the two nodes share their address arithmetic (the second node's global accesses are the
// first's plus 32 elements), and the shared tiles hold the two columns of a thread side by
// side (PairTile), so that every stencil access of both nodes is one 8-byte shared load.
// The one-node kernel is bound by instruction issue; this one issues about 40% fewer
// instructions per node.  The arithmetic per node is the one-node kernel's, operation for
// operation, each rounded once, so the two give identical bits (as do the bulk-copy and
// batch kernels, which run the one-node phases).
//
// Phases (as in fused_step):
//   phase 1  pull the 9N values of both owned nodes (plane base addresses from the launch
//            parameters), sum rho_i and the first moment, rho~_i, ln f_i; the 2-node halo
//            ring of the 64-wide tile (304 nodes for 8 rows) is pulled two ring nodes per
//            thread for rho~ only, with ln f on its inner row;
//   phase 2  Phi_i = sum_j kappa_ij lap rho~_j - RT ln f_i on every pair slot of the tile + 1
//            box;
//   phase 3  force, velocity, equilibrium, forcing and collision per node pair, coalesced
//            stores at the nodes (streaming happens on the next step's read side).
// The last NPARK components' pulled values wait in shared memory between phases 1 and 3.
// LAG: the lagged reading of the velocity (a launch with A.lagged set).
// A pending diagnostics request is served as in fused_step: the partial sums of each 32 x 8
// strip go where reduce_partial would put them, bit for bit.
#pragma once

#include "fmlbm_kernels.cuh"


namespace fmlbm {

constexpr int kPW = 2 * kTX;  // width of the paired tile

template <int NC, int TY>
struct PairSmem {
    PairTile<NC, TY, 2> rt;     // rho~ on tile + 2
    PairTile<NC, TY, 1> lf;     // ln f on tile + 1
    PairTile<NC, TY, 1> G;      // Phi_i on tile + 1
    float2 Fl[2][TY][kTX];      // stored total force at the tile's node pairs (lagged reading)
};

// Ring nodes of the paired tile (two per thread of the first RING / 2 threads).
template <int TY> constexpr int kPairRing = 4 * (kPW + 4) + 4 * TY;

// The park area: the parked values, five 16-byte slots per parked component and thread.
template <int NC, int ST, int TY, int NPARK>
constexpr size_t pair_park_bytes() {
    return (size_t)NPARK * 5 * 16 * kTX * TY;
}
// Shared bytes of the paired step: the tiles, the park area, the diagnostics snapshot copy
// of the tile's node pairs.
template <int NC, int ST, int TY, int NPARK>
constexpr size_t pair_smem_bytes() {
    return sizeof(PairSmem<NC, TY>) + pair_park_bytes<NC, ST, TY, NPARK>() + (size_t)NC * TY * kTX * 8;
}

// One column's value into a pair tile: into the slot where it is lane 0 and, for the 2H
// columns held twice, into the slot where it is lane 1.  col: tile column, -H .. 63 + H.
template <int NC, int TY, int H>
__device__ __forceinline__ void pair_put(PairTile<NC, TY, H>& t, int i, int row, int col, float v) {
    if (col < kTX + H) t.v[i][row][col + H].x = v;
    if (col >= kTX - H) t.v[i][row][col - kTX + H].y = v;
}
// A thread's node pair (columns c and c + 32, c = 0 .. 31) into a pair tile.
template <int NC, int TY, int H>
__device__ __forceinline__ void pair_put2(PairTile<NC, TY, H>& t, int i, int row, int c, float2 v) {
    t.v[i][row][c + H] = v;
    if (c >= kTX - H) t.v[i][row][c - kTX + H].y = v.x;
    if (c < H) t.v[i][row][c + kTX + H].x = v.y;
}

// Parked values of one component: slots k = 0..3 hold (h[2k], h[2k+1]) of both lanes as
// float4 (h[2k].x, h[2k].y, h[2k+1].x, h[2k+1].y); slot 4 holds h[8].
__device__ __forceinline__ void park_pair_store(const float2 (&h)[9], float4* park, int tid, int NT) {
#pragma unroll
    for (int k = 0; k < 4; ++k) park[k * NT + tid] = make_float4(h[2 * k].x, h[2 * k].y, h[2 * k + 1].x, h[2 * k + 1].y);
    reinterpret_cast<float2*>(park + 4 * NT)[2 * tid] = h[8];
}
__device__ __forceinline__ void park_pair_load(float2 (&h)[9], const float4* park, int tid, int NT) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float4 v = park[k * NT + tid];
        h[2 * k] = make_float2(v.x, v.y);
        h[2 * k + 1] = make_float2(v.z, v.w);
    }
    h[8] = reinterpret_cast<const float2*>(park + 4 * NT)[2 * tid];
}

// Pulled sums of two nodes (wx0, wy0), (wx1, wy1) (wrapped coordinates), in direction order.
template <int NC, int ST>
__device__ __forceinline__ void pull_rho_pair(const Planes& P, int wx0, int wy0, int wx1, int wy1, bool inner, int nx,
                                              int ny, float2* rs) {
    auto src_of = [&](int a, int wx, int wy) {
        if (inner) return wy * nx + wx - ey(a) * nx - ex(a);
        const int xm = wx == 0 ? nx - 1 : wx - 1, xp = wx == nx - 1 ? 0 : wx + 1;
        const int ym = wy == 0 ? ny - 1 : wy - 1, yp = wy == ny - 1 ? 0 : wy + 1;
        return pull_src(a, wx, wy, xm, xp, ym, yp, nx);
    };
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        const int s0 = src_of(a, wx0, wy0), s1 = src_of(a, wx1, wy1);
#pragma unroll
        for (int i = 0; i < NC; ++i) {
            const float2 v = make_float2(load_gp<ST>(P, i, a, s0), load_gp<ST>(P, i, a, s1));
            rs[i] = a == 0 ? v : vadd(rs[i], v);
        }
    }
}

template <int NC, int ST, int TY, int NPARK, bool LAG>
__global__ void __launch_bounds__(kTX* TY, NPARK > 0 ? 4 : 3) fused_step_pair(StepArgs A, Planes P) {
    static_assert(ST != ST_F64, "the paired step packs float arithmetic");
    static_assert(NPARK >= 0 && NPARK <= NC, "parked components");
    static_assert(TY == 8, "the phase-2 work split below assumes 8 rows");
    using V = float2;
    constexpr int NT = kTX * TY;
    constexpr int NREG = NC - NPARK;  // components whose pulled values stay in registers
    static_assert(sizeof(PairSmem<NC, TY>) % 16 == 0, "the parked values are 16-byte slots");
    extern __shared__ __align__(16) unsigned char smem_pair[];
    auto& S = *reinterpret_cast<PairSmem<NC, TY>*>(smem_pair);
    float4* park = reinterpret_cast<float4*>(smem_pair + sizeof(PairSmem<NC, TY>));
    float2* pv_s = reinterpret_cast<float2*>(smem_pair + sizeof(PairSmem<NC, TY>) + pair_park_bytes<NC, ST, TY, NPARK>());
    const MixConstT<float>& m = A.mixf;
    const int nx = A.nx, ny = A.ny, nxy = nx * ny;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kTX + tx;
    const int x0 = blockIdx.x * kPW, y0 = blockIdx.y * TY;
    const bool inner = x0 >= 3 && x0 + kPW + 3 <= nx && y0 >= 3 && y0 + TY + 3 <= ny;
    const int gx0 = x0 + tx, gx1 = gx0 + kTX, gy = y0 + ty;
    const bool valid0 = gx0 < nx && gy < ny, valid1 = gx1 < nx && gy < ny;
    const unsigned vmask = (valid0 ? 1u : 0u) | (valid1 ? 2u : 0u);
    const bool diag = A.diag_partial != nullptr;

    // the stored force F(t - 1) and the diagnostics snapshot of the owned nodes, copied into
    // shared memory while phases 1-2 run (cp.async)
    {
        const float* Fin = static_cast<const float*>(A.Fin);
        const float* prev = static_cast<const float*>(A.rho_prev);
        if (valid0) {
            const int node = gy * nx + gx0;
            if (LAG) {
                cp_async_elem(&S.Fl[0][ty][tx].x, Fin + node);
                cp_async_elem(&S.Fl[1][ty][tx].x, Fin + nxy + node);
            }
            if (diag)
#pragma unroll
                for (int i = 0; i < NC; ++i) cp_async_elem(&pv_s[(i * TY + ty) * kTX + tx].x, prev + (size_t)i * nxy + node);
        }
        if (valid1) {
            const int node = gy * nx + gx1;
            if (LAG) {
                cp_async_elem(&S.Fl[0][ty][tx].y, Fin + node);
                cp_async_elem(&S.Fl[1][ty][tx].y, Fin + nxy + node);
            }
            if (diag)
#pragma unroll
                for (int i = 0; i < NC; ++i) cp_async_elem(&pv_s[(i * TY + ty) * kTX + tx].y, prev + (size_t)i * nxy + node);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }

    // ---- phase 1: the ring pair (pull, rho~, ln f on the inner ring), then the owned nodes
    //      (pull, rho_i and the first moment, the parked components to shared memory, rho~ and
    //      ln f), so that only one set of pulled values is live at a time.  (The ring's values
    //      copied into shared memory by cp.async, so that their latency would overlap the
    //      owned pulls, measured slower: the registers then spill.) ----
    constexpr int RING = kPairRing<TY>;
    constexpr int RP = RING / 2;
    static_assert(RING % 2 == 0 && RP <= NT, "two ring nodes per thread at most");
    const bool has_ring = tid < RP;
    int bx0 = 0, by0 = 0, bx1 = 0, by1 = 0;
    V rr[NC];
    if (has_ring) {
        ring_position<TY, kPW>(tid, bx0, by0);
        ring_position<TY, kPW>(tid + RP, bx1, by1);
        const int wx0 = inner ? x0 - 2 + bx0 : wrap(x0 - 2 + bx0, nx);
        const int wy0 = inner ? y0 - 2 + by0 : wrap(y0 - 2 + by0, ny);
        const int wx1 = inner ? x0 - 2 + bx1 : wrap(x0 - 2 + bx1, nx);
        const int wy1 = inner ? y0 - 2 + by1 : wrap(y0 - 2 + by1, ny);
        pull_rho_pair<NC, ST>(P, wx0, wy0, wx1, wy1, inner, nx, ny, rr);
#pragma unroll
        for (int i = 0; i < NC; ++i) {
            rr[i] = vmul(rr[i], vbc<V>(m.invM[i]));
            pair_put(S.rt, i, by0, bx0 - 2, rr[i].x);
            pair_put(S.rt, i, by1, bx1 - 2, rr[i].y);
        }
        const bool in0 = bx0 >= 1 && bx0 <= kPW + 2 && by0 >= 1 && by0 <= TY + 2;
        const bool in1 = bx1 >= 1 && bx1 <= kPW + 2 && by1 >= 1 && by1 <= TY + 2;
        if (in0 || in1) {
            V lnf[NC];
            node_lnf<NC, V>(m, rr, lnf);
#pragma unroll
            for (int i = 0; i < NC; ++i) {
                if (in0) pair_put(S.lf, i, by0 - 1, bx0 - 2, lnf[i].x);
                if (in1) pair_put(S.lf, i, by1 - 1, bx1 - 2, lnf[i].y);
            }
        }
    }
    V g[NREG > 0 ? NREG : 1][9];
    V r[NC], jx, jy;
    {
        V gp[NC][9];
        const int wx0 = inner ? gx0 : wrap(gx0, nx), wx1 = inner ? gx1 : wrap(gx1, nx);
        const int wy = inner ? gy : wrap(gy, ny);
        if (inner) {
            // both nodes inside: the second node's source is the first's plus 32 elements
            const int node = wy * nx + wx0;
#pragma unroll
            for (int a = 0; a < 9; ++a) {
                const int src = node - ey(a) * nx - ex(a);
#pragma unroll
                for (int i = 0; i < NC; ++i)
                    gp[i][a] = make_float2(load_gp<ST>(P, i, a, src), load_gp<ST>(P, i, a, src + kTX));
            }
        } else {
            const int ym = wy == 0 ? ny - 1 : wy - 1, yp = wy == ny - 1 ? 0 : wy + 1;
            const int xm0 = wx0 == 0 ? nx - 1 : wx0 - 1, xp0 = wx0 == nx - 1 ? 0 : wx0 + 1;
            const int xm1 = wx1 == 0 ? nx - 1 : wx1 - 1, xp1 = wx1 == nx - 1 ? 0 : wx1 + 1;
#pragma unroll
            for (int a = 0; a < 9; ++a) {
                const int s0 = pull_src(a, wx0, wy, xm0, xp0, ym, yp, nx);
                const int s1 = pull_src(a, wx1, wy, xm1, xp1, ym, yp, nx);
#pragma unroll
                for (int i = 0; i < NC; ++i)
                    gp[i][a] = make_float2(load_gp<ST>(P, i, a, s0), load_gp<ST>(P, i, a, s1));
            }
        }
#pragma unroll
        for (int i = 0; i < NC; ++i) {
            r[i] = sum9(gp[i]);
            moment_j(gp[i], i == 0, jx, jy);
        }
#pragma unroll
        for (int c = 0; c < NPARK; ++c) park_pair_store(gp[NREG + c], park + c * 5 * NT, tid, NT);
#pragma unroll
        for (int i = 0; i < NREG; ++i)
#pragma unroll
            for (int a = 0; a < 9; ++a) g[i][a] = gp[i][a];
    }
    {
        V rt[NC], lnf[NC];
#pragma unroll
        for (int i = 0; i < NC; ++i) {
            rt[i] = vmul(r[i], vbc<V>(m.invM[i]));
            pair_put2(S.rt, i, ty + 2, tx, rt[i]);
        }
        const V beta = node_lnf<NC, V>(m, rt, lnf);
#pragma unroll
        for (int i = 0; i < NC; ++i) pair_put2(S.lf, i, ty + 1, tx, lnf[i]);
        domain_check<NC, V>(A, rt, lnf, beta, gx0, kTX, gy, checked_row(A, gy) ? vmask : 0u);
    }
    __syncthreads();

    // ---- phase 2 on the 34 pair slots of each of the TY + 2 rows of the tile + 1 box:
    //      warp w takes slots 0..31 of row w; rows TY, TY + 1 go to the last two warps and
    //      slots 32, 33 of every row to warp TY - 3 (the ring ran on the first warps) ----
    phase2_core<NC, V>(m, S.rt, S.lf, S.G, A.stencil, tx, ty, 0);
    if (ty >= TY - 2) phase2_core<NC, V>(m, S.rt, S.lf, S.G, A.stencil, tx, ty + 2, 0);
    if (ty == TY - 3 && tx < 2 * (TY + 2))
        phase2_core<NC, V>(m, S.rt, S.lf, S.G, A.stencil, kTX + (tx & 1), tx >> 1, 0);
    __syncthreads();

    // ---- phase 3 ----
    if (valid0) {  // valid1 implies valid0
        V Fpx = vbc<V>(0.f), Fpy = vbc<V>(0.f);
        if constexpr (LAG) {
            asm volatile("cp.async.wait_all;\n" ::: "memory");
            Fpx = S.Fl[0][ty][tx];
            Fpy = S.Fl[1][ty][tx];
        }
        auto geth = [&](int i, V (&h)[9]) {
            if (i >= NREG) {
                park_pair_load(h, park + (i - NREG) * 5 * NT, tid, NT);
            } else {
#pragma unroll
                for (int a = 0; a < 9; ++a) h[a] = g[i][a];
            }
        };
        const int node0 = gy * nx + gx0;
        auto store = [&](int i, int a, V v) {
            store_gp<ST>(P, i, a, node0, v.x);
            if (valid1) store_gp<ST>(P, i, a, node0 + kTX, v.y);
        };
        V Ftx, Fty, ux, uy;
        phase3_core<NC, true, false, LAG, V>(m, A.stencil, S.G, S.rt, tx + 1, ty + 1, 0, r, jx, jy, geth, Fpx, Fpy,
                                             store, Ftx, Fty, ux, uy);
        float* Fout = static_cast<float*>(A.Fout);
        Fout[node0] = Ftx.x;
        Fout[nxy + node0] = Fty.x;
        if (valid1) {
            Fout[node0 + kTX] = Ftx.y;
            Fout[nxy + node0 + kTX] = Fty.y;
        }
    }

    // ---- diagnostics of the state this step read (uniform in diag) ----
    if (diag) {
        static_assert(TY % 8 == 0, "diagnostics strips of 8 rows");
        __shared__ Sum2<V> dred[TY][NC + 2];
        Sum2<V> acc[NC + 2];
#pragma unroll
        for (int k = 0; k < NC + 2; ++k) acc[k] = s2_of(vbc<V>(0.f));
        if (valid0) {
            asm volatile("cp.async.wait_all;\n" ::: "memory");
            V pv[NC];
#pragma unroll
            for (int i = 0; i < NC; ++i) pv[i] = pv_s[(i * TY + ty) * kTX + tx];
            diag_node<NC, V>(r, pv, A.have_prev, acc);
            if (!valid1)
#pragma unroll
                for (int k = 0; k < NC + 2; ++k) acc[k].hi.y = acc[k].lo.y = 0.f;
            float* prev = static_cast<float*>(A.rho_prev);
            const int node0 = gy * nx + gx0;
#pragma unroll
            for (int i = 0; i < NC; ++i) {
                prev[(size_t)i * nxy + node0] = r[i].x;
                if (valid1) prev[(size_t)i * nxy + node0 + kTX] = r[i].y;
            }
        }
        diag_warp<NC, V>(acc, dred[ty]);
        __syncthreads();
        constexpr int STRIPS = TY / 8;
        const int tiles_x = (nx + kTX - 1) / kTX;
        if (tid < 2 * STRIPS * (NC + 2)) {
            const int half = tid / (STRIPS * (NC + 2)), q = tid % (STRIPS * (NC + 2));
            const int sub = q / (NC + 2), k = q % (NC + 2);
            const int col = 2 * blockIdx.x + half;
            if (col < tiles_x && y0 + 8 * sub < ny)
                static_cast<double*>(A.diag_partial)[((size_t)(blockIdx.y * STRIPS + sub) * tiles_x + col) * (NC + 2) +
                                                     k] = diag_strip<NC, V>(dred, 8 * sub, k, half);
        }
    }
}

}  // namespace fmlbm
