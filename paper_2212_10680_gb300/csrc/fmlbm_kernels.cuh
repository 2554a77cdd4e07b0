// Device code of libfmlbm: the fused lattice update and its helpers (sm_103a).
//
// One launch of `fused_step` performs one full time step of the fugacity-based
// free-energy LBM (Section III.B, steps 1-9) for every node of a lattice:
//
//   phase 1  pull the 9N post-collision values of the previous step into
//            registers (streaming, step 9 of the previous step), sum them to
//            rho_i (step 1) and rho~_i = rho_i / M_i (step 2), and evaluate the
//            mixing rules, pressure and ln f_i (steps 3-5, the density-explicit
//            form of Eq. eqfugupdatePR/SRK/VDW); the same on a 2-node halo ring
//            (rho~ to shared memory, ln f on its inner row);
//   phase 2  on the tile plus a 1-node halo: Phi_i = sum_j kappa_ij lap(rho~_j)
//            - RT ln f_i (step 6 with mu_I,i = -sum_j kappa_ij lap rho~_j);
//   phase 3  at each node: F_i = rho~_i grad Phi_i, which is Eq. eqforcefinal
//            (step 7; the stencils are linear), u from the first moment and half
//            the force (step 1), g^eq (Eq. eqLBEMCb, rho_0 = 0) and F_{a,i}
//            (Eq. eqLBEMCfinal3) (step 8), BGK collision (Eq. eqLBEMCa), and a
//            coalesced store of the post-collision values at the node itself
//            (the next launch pulls them: streaming happens on the read side).
//
// The per-node arithmetic is written once over a lane type (fmlbm_lanes.cuh): one node
// per thread here, two nodes per thread in the paired step (fmlbm_pair.cuh), with every
// operation rounded once and never contracted, so all kernels give the same bits.
//
// Everything between the one read and the one write of the distributions
// stays on chip; the only other global traffic is the stored total force
// sum_i F_i (2 values per node) used by the next step's velocity, and, when a
// diagnostics request is pending, the density snapshot and per-strip sums of
// the state the step reads.  With two components in float storage the second
// component's pulled values wait in shared memory between phases 1 and 3 and
// the distribution planes are addressed through a second launch parameter
// (Planes), so that the step fits 48 registers (five blocks per SM).
//
// Buffer layout (structure of arrays): plane (i, a) of the distributions is a
// contiguous nx*ny array in row-major (y, x) order; plane index i*9 + a for
// FP64/FP32 storage.  In the 16-bit deviation forms g_0 planes are float
// ([N][ny][nx]) and g_a, a = 1..8, planes are 16-bit ([N][8][ny][nx]).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "fmlbm_lanes.cuh"

namespace fmlbm {

constexpr int kMaxC = 4;
constexpr int kTX = 32;  // tile width = one warp

// Storage forms of the kernels.  The _X forms store like the 16-bit forms and evaluate the
// fugacity terms of ln f in double (node_lnf_st).
enum Storage { ST_F64 = 0, ST_F32 = 1, ST_F16DEV = 2, ST_BF16DEV = 3, ST_F16DEV_X = 4, ST_BF16DEV_X = 5 };
template <int ST> constexpr bool kDev16 = ST == ST_F16DEV || ST == ST_BF16DEV || ST == ST_F16DEV_X || ST == ST_BF16DEV_X;
template <int ST> constexpr bool kLnf64 = ST == ST_F16DEV_X || ST == ST_BF16DEV_X;

// D2Q9: a = 0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1) 5:(1,1) 6:(-1,1) 7:(-1,-1) 8:(1,-1)
__host__ __device__ __forceinline__ constexpr int ex(int a) {
    return (a == 1 || a == 5 || a == 8) ? 1 : ((a == 3 || a == 6 || a == 7) ? -1 : 0);
}
__host__ __device__ __forceinline__ constexpr int ey(int a) {
    return (a == 2 || a == 5 || a == 6) ? 1 : ((a == 4 || a == 7 || a == 8) ? -1 : 0);
}
template <typename R>
__host__ __device__ __forceinline__ constexpr R wgt(int a) {
    return a == 0 ? R(4) / R(9) : (a < 5 ? R(1) / R(9) : R(1) / R(36));
}

// Mixture constants, computed on the host from Appendix C (T fixed).  Kernels read
// the copy in their own arithmetic type (no double -> float conversions on device,
// which would run on the FP64 pipe).
template <typename E>
struct MixConstT {
    int nc;
    int eos;          // 0 PR, 1 SRK, 2 vdW
    E RT;
    E b[kMaxC];
    E M[kMaxC];
    E invM[kMaxC];
    E aij[kMaxC * kMaxC];   // (a alpha)_ij, row stride kMaxC
    E kap[kMaxC * kMaxC];   // kappa_ij = sqrt(kappa_i kappa_j), row stride kMaxC
    E omega;                // 1 / tau
    E fcoef;                // 1 - 1 / (2 tau)
    E invRT;                // 1 / (R T)
};
using MixConst = MixConstT<double>;

template <typename E>
MixConstT<E> cast_mix(const MixConst& m) {
    MixConstT<E> r;
    r.nc = m.nc;
    r.eos = m.eos;
    r.RT = (E)m.RT;
    for (int i = 0; i < kMaxC; ++i) {
        r.b[i] = (E)m.b[i];
        r.M[i] = (E)m.M[i];
        r.invM[i] = (E)m.invM[i];
    }
    for (int k = 0; k < kMaxC * kMaxC; ++k) {
        r.aij[k] = (E)m.aij[k];
        r.kap[k] = (E)m.kap[k];
    }
    r.omega = (E)m.omega;
    r.fcoef = (E)m.fcoef;
    r.invRT = (E)m.invRT;
    return r;
}

struct ErrorLatch {
    int flag;         // 0 = clean, 1 = a node left the EOS domain, 2 = a bounded wait ran out
    int comp, x, y;
};

struct StepArgs {
    int nx, ny;
    int stencil;      // 0 isotropic, 1 central
    int lagged;       // 1: u uses the stored force of the previous step
    int standard;     // 1: standard formulation (Eq. eqLBE, force of Eq. eqForceGen)
    const void* gin;  // F64/F32: all planes; DEV: 16-bit planes a = 1..8
    const float* g0in;  // DEV: float planes a = 0
    void* gout;
    float* g0out;
    const void* Fin;  // [2][ny][nx] Real
    void* Fout;
    // moments mode outputs (double, may be null)
    double* rho_out;
    double* u_out;
    double* lnf_out;
    ErrorLatch* err;
    MixConstT<double> mixd;
    MixConstT<float> mixf;
    // diagnostics of the input state fused into a plain step (diag_partial null: none):
    // N + 2 sums per 32 x 8 strip in reduce_partial's layout (storage arithmetic type),
    // and the density snapshot
    void* diag_partial;
    void* rho_prev;  // [N][ny][nx] in the storage arithmetic type
    int have_prev;
    // rows [check_y0, check_y1) whose nodes the domain check covers (check_y1 = 0: all); a slab
    // of a decomposed lattice leaves out its ghost rows, whose update is discarded
    int check_y0, check_y1;
    int pad0;
    long long wait_polls;  // polls of a bounded wait for a tile copy (bulk-copy step forms)
};
__device__ __forceinline__ bool checked_row(const StepArgs& A, int y) {
    return A.check_y1 == 0 || (y >= A.check_y0 && y < A.check_y1);
}

// The base address of every distribution plane of A.gin / A.gout, a second launch
// parameter of the single-lattice step only (in StepArgs it made the batch kernel, which
// copies each lattice's StepArgs into shared memory per tile, 7% slower on the serving
// workload).  F64/F32 storage: plane i*9+a; 16-bit storage: plane i*8+a-1 (a >= 1) and
// float plane i (a = 0).  The launcher fills it from A (make_planes).
struct Planes {
    const void* in[kMaxC * 9];
    void* out[kMaxC * 9];
    const float* g0in[kMaxC];
    float* g0out[kMaxC];
};

// elem: bytes per element of the planes A.gin / A.gout point to (8, 4 or 2); unused entries
// and those of null buffers stay null.
inline Planes make_planes(const StepArgs& A, int nc, bool dev16, size_t elem) {
    Planes P = {};
    const size_t nxy = (size_t)A.nx * A.ny;
    const int per = dev16 ? 8 : 9;
    for (int k = 0; k < nc * per; ++k) {
        P.in[k] = A.gin ? static_cast<const char*>(A.gin) + k * nxy * elem : nullptr;
        P.out[k] = A.gout ? static_cast<char*>(A.gout) + k * nxy * elem : nullptr;
    }
    for (int i = 0; i < nc && dev16; ++i) {
        P.g0in[i] = A.g0in ? A.g0in + i * nxy : nullptr;
        P.g0out[i] = A.g0out ? A.g0out + i * nxy : nullptr;
    }
    return P;
}

template <typename E> __device__ __forceinline__ const MixConstT<E>& mixc(const StepArgs& A);
template <> __device__ __forceinline__ const MixConstT<double>& mixc<double>(const StepArgs& A) { return A.mixd; }
template <> __device__ __forceinline__ const MixConstT<float>& mixc<float>(const StepArgs& A) { return A.mixf; }

template <int ST> struct StoreTraits;
template <> struct StoreTraits<ST_F64> { using Real = double; using Elem = double; };
template <> struct StoreTraits<ST_F32> { using Real = float; using Elem = float; };
template <> struct StoreTraits<ST_F16DEV> { using Real = float; using Elem = __half; };
template <> struct StoreTraits<ST_BF16DEV> { using Real = float; using Elem = __nv_bfloat16; };
template <> struct StoreTraits<ST_F16DEV_X> { using Real = float; using Elem = __half; };
template <> struct StoreTraits<ST_BF16DEV_X> { using Real = float; using Elem = __nv_bfloat16; };

__device__ __forceinline__ float to_real(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_real(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_real(float v) { return v; }
__device__ __forceinline__ double to_real(double v) { return v; }
template <typename E> __device__ __forceinline__ E from_real(float v);
template <> __device__ __forceinline__ __half from_real<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_real<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <> __device__ __forceinline__ float from_real<float>(float v) { return v; }

// Read-only loads through the non-coherent path.
template <typename E> __device__ __forceinline__ E ldg(const E* p) { return __ldg(p); }
template <> __device__ __forceinline__ __half ldg<__half>(const __half* p) { return __ldg(p); }
template <> __device__ __forceinline__ __nv_bfloat16 ldg<__nv_bfloat16>(const __nv_bfloat16* p) {
    return __ldg(p);
}

template <int ST>
__device__ __forceinline__ typename StoreTraits<ST>::Real load_g(const StepArgs& A, int i, int a, size_t node,
                                                                  size_t nxy) {
    using Elem = typename StoreTraits<ST>::Elem;
    if constexpr (ST == ST_F64 || ST == ST_F32) {
        return to_real(ldg(static_cast<const Elem*>(A.gin) + (size_t)(i * 9 + a) * nxy + node));
    } else {
        if (a == 0) return ldg(A.g0in + (size_t)i * nxy + node);
        return to_real(ldg(static_cast<const Elem*>(A.gin) + (size_t)(i * 8 + a - 1) * nxy + node));
    }
}

// Loads cached in L2 only (ld.global.cg), for data that other multiprocessors write during the
// same launch (the multi-step kernel): the L1 of this multiprocessor may hold stale copies.
template <typename E> __device__ __forceinline__ E ldcg(const E* p) { return __ldcg(p); }
template <> __device__ __forceinline__ __half ldcg<__half>(const __half* p) {
    const unsigned short b = __ldcg(reinterpret_cast<const unsigned short*>(p));
    return __ushort_as_half(b);
}
template <> __device__ __forceinline__ __nv_bfloat16 ldcg<__nv_bfloat16>(const __nv_bfloat16* p) {
    const unsigned short b = __ldcg(reinterpret_cast<const unsigned short*>(p));
    return __ushort_as_bfloat16(b);
}
template <bool CG, typename E> __device__ __forceinline__ E ldsel(const E* p) {
    if constexpr (CG) return ldcg(p);
    else return ldg(p);
}

// The same through the plane base addresses of the launch's parameters and a 32-bit node
// index: each access address is then a single multiply-add onto a parameter, where the
// forms above compute a 64-bit plane offset (two-component step: +1.5% on GB300; with
// three components it cost registers and spilled).  CG: L2-only loads (ldcg).
template <int ST, bool CG = false>
__device__ __forceinline__ typename StoreTraits<ST>::Real load_gp(const Planes& P, int i, int a, int node) {
    using Elem = typename StoreTraits<ST>::Elem;
    if constexpr (ST == ST_F64 || ST == ST_F32) {
        return to_real(ldsel<CG>(static_cast<const Elem*>(P.in[i * 9 + a]) + node));
    } else {
        if (a == 0) return ldsel<CG>(P.g0in[i] + node);
        return to_real(ldsel<CG>(static_cast<const Elem*>(P.in[i * 8 + a - 1]) + node));
    }
}
template <int ST>
__device__ __forceinline__ void store_gp(const Planes& P, int i, int a, int node, typename StoreTraits<ST>::Real v) {
    using Elem = typename StoreTraits<ST>::Elem;
    if constexpr (ST == ST_F64 || ST == ST_F32) {
        static_cast<Elem*>(P.out[i * 9 + a])[node] = v;
    } else {
        if (a == 0)
            P.g0out[i][node] = v;
        else
            static_cast<Elem*>(P.out[i * 8 + a - 1])[node] = from_real<Elem>(v);
    }
}

template <int ST>
__device__ __forceinline__ void store_g(const StepArgs& A, int i, int a, size_t node, size_t nxy,
                                        typename StoreTraits<ST>::Real v) {
    using Elem = typename StoreTraits<ST>::Elem;
    if constexpr (ST == ST_F64) {
        static_cast<double*>(A.gout)[(size_t)(i * 9 + a) * nxy + node] = v;
    } else if constexpr (ST == ST_F32) {
        static_cast<float*>(A.gout)[(size_t)(i * 9 + a) * nxy + node] = v;
    } else {
        if (a == 0)
            A.g0out[(size_t)i * nxy + node] = v;
        else
            static_cast<Elem*>(A.gout)[(size_t)(i * 8 + a - 1) * nxy + node] = from_real<Elem>(v);
    }
}

template <int ST, bool PP>
__device__ __forceinline__ void store_gsel(const StepArgs& A, const Planes* P, int i, int a, int node, int nxy,
                                           typename StoreTraits<ST>::Real v) {
    if constexpr (PP) store_gp<ST>(*P, i, a, node, v);
    else store_g<ST>(A, i, a, (size_t)node, (size_t)nxy, v);
}

__device__ __forceinline__ int wrap(int v, int n) {
    int r = v % n;
    return r < 0 ? r + n : r;
}

// ln f_i at one node from its molar densities (steps 2-5), written in terms of the
// packing fraction beta = b_m rho~ so that v = 1 / rho~ never appears:
//   ln x_i - ln((v - b_m)/RT) = ln(rho~_i RT / (1 - beta))
//   PR : p v / RT - 1 = beta/(1-beta) - (aa_m rho~ / RT) / (1 + 2 beta - beta^2)
//        ln[(v + (1+sqrt2) b_m)/(v + (1-sqrt2) b_m)] = ln[(1 + (1+sqrt2) beta)/(1 + (1-sqrt2) beta)]
//   SRK: p v / RT - 1 = beta/(1-beta) - (aa_m rho~ / RT) / (1 + beta),  ln(1 + b_m / v) = log1p(beta)
//   vdW: b_i / (v - b_m) = b_i rho~ / (1 - beta),  2 S_i / (RT v) = 2 S_i rho~ / RT
// (each logarithm takes a ratio whose relative rounding is a few ulp, so merging the
// printed logarithms pairwise costs no accuracy).  Lane arithmetic: one node per lane.
// Returns beta (for the domain check).  eos >= 0: that EOS (a constant the caller passes, so
// that the branches below fold away); -1: the mixture's.
template <int NC, typename V, typename E>
__device__ __forceinline__ V node_lnf(const MixConstT<E>& m, const V* rt, V* lnf, int eos = -1) {
    const int kind = eos >= 0 ? eos : m.eos;
    V rtot = rt[0];
#pragma unroll
    for (int i = 1; i < NC; ++i) rtot = vadd(rtot, rt[i]);
    const V inv = vrcp(rtot);
    V beta = vmul(vbc<V>(m.b[0]), rt[0]);  // b_m rho~ = sum_i b_i rho~_i (the packing fraction)
#pragma unroll
    for (int i = 1; i < NC; ++i) beta = vfma(vbc<V>(m.b[i]), rt[i], beta);
    V S[NC];                               // rho~ S_i = sum_j (a alpha)_ij rho~_j
    V aam_rt2;                             // (a alpha)_m rho~^2
#pragma unroll
    for (int i = 0; i < NC; ++i) {
        V s = vmul(vbc<V>(m.aij[i * kMaxC]), rt[0]);
#pragma unroll
        for (int j = 1; j < NC; ++j) s = vfma(vbc<V>(m.aij[i * kMaxC + j]), rt[j], s);
        S[i] = s;
        aam_rt2 = i == 0 ? vmul(rt[0], s) : vfma(rt[i], s, aam_rt2);
    }
    const V one = vbc<V>(E(1));
    const V invomb = vrcp(vsub(one, beta));
    const V lead = vmul(vbc<V>(m.RT), invomb);
    if (kind == 2) {
        const V rb1 = vmul(rtot, invomb);               // rho~ / (1 - beta)
        const V m2rt = vbc<V>(E(-2) * m.invRT);
#pragma unroll
        for (int i = 0; i < NC; ++i)
            lnf[i] = vfma(S[i], m2rt, vfma(vbc<V>(m.b[i]), rb1, vln(vmul(rt[i], lead))));
        return beta;
    }
    const V att = vmul(vmul(aam_rt2, inv), vbc<V>(m.invRT));   // (a alpha)_m rho~ / RT
    V rep, lr;
    E pref;
    if (kind == 0) {
        const E s2 = E(1.4142135623730950488);
        const V den = vfma(beta, vsub(vbc<V>(E(2)), beta), one);   // 1 + 2 beta - beta^2
        rep = vfma(vneg(att), vrcp(den), vmul(beta, invomb));
        lr = vln(vmul(vfma(vbc<V>(E(1) + s2), beta, one), vrcp(vfma(vbc<V>(E(1) - s2), beta, one))));
        pref = m.invRT * E(0.35355339059327376220);  // 1 / (2 sqrt2 RT)
    } else {
        rep = vfma(vneg(att), vrcp(vadd(one, beta)), vmul(beta, invomb));
        lr = vlog1p(beta);
        pref = m.invRT;
    }
    // with b_m = beta / rho~ the coefficient of lr, ((a alpha)_m b_i/b_m - 2 sum_j x_j (a alpha)_ij)
    // / (c b_m RT), becomes pref ((a alpha)_m b_i/b_m - 2 S_i / rho~) rho~ / beta
    const V rb = vmul(rtot, vrcp(beta));                       // 1 / b_m
    const V aam = vmul(vmul(aam_rt2, inv), inv);               // (a alpha)_m
    const V plr = vmul(vmul(vbc<V>(pref), rb), lr);
    const V m2inv = vmul(vbc<V>(E(-2)), inv);
#pragma unroll
    for (int i = 0; i < NC; ++i) {
        const V bi = vmul(vbc<V>(m.b[i]), rb);                 // b_i / b_m
        const V t = vfma(aam, bi, vmul(S[i], m2inv));          // (a alpha)_m b_i/b_m - 2 S_i / rho~
        lnf[i] = vfma(plr, t, vfma(bi, rep, vln(vmul(rt[i], lead))));
    }
    return beta;
}

// Shared-memory tile of a field with a halo of H nodes around TW x TY nodes.
template <typename E, int NC, int TY, int H, int TW = kTX>
struct Tile {
    static constexpr int W = TW + 2 * H;
    static constexpr int Hh = TY + 2 * H;
    E v[NC][Hh][W];
};

// ln f of a node in the storage form's arithmetic: float (or double) lanes as node_lnf; the
// _X forms evaluate the fugacity terms (mixing sums, the repulsion and attraction terms and
// their logarithms) in double from the float densities, with the double mixture constants,
// and round ln f and beta to float once.
template <int NC, bool LNF64, typename Real>
__device__ __forceinline__ Real node_lnf_st(const StepArgs& A, const MixConstT<Real>& m, const Real* rt, Real* lnf,
                                            int eos = -1) {
    if constexpr (LNF64) {
        double rd[NC], ld[NC];
#pragma unroll
        for (int i = 0; i < NC; ++i) rd[i] = (double)rt[i];
        const double beta = node_lnf<NC, double>(A.mixd, rd, ld, eos);
#pragma unroll
        for (int i = 0; i < NC; ++i) lnf[i] = (Real)ld[i];
        return (Real)beta;
    } else {
        return node_lnf<NC, Real>(m, rt, lnf, eos);
    }
}

// A field on a 64 x TY tile plus an H-node halo, stored in pair slots for the paired step:
// slot s of a row holds the columns (s - H, s - H + 32) of the tile (column 0 = the tile's
// first) as one float2, so that a thread's two nodes, and the same neighbour of both, are
// one 8-byte access.  Lane 0 of the slots covers columns -H .. 31 + H, lane 1 columns
// 32 - H .. 63 + H; the 2H columns 32 - H .. 31 + H appear in two slots.  Slot and row
// indices are the tile coordinates of the one-node tiles (column + H, row + H).
template <int NC, int TY, int H>
struct PairTile {
    static constexpr int S = kTX + 2 * H;
    static constexpr int R = TY + 2 * H;
    static constexpr int halo = H;
    float2 v[NC][R][S];
};
template <typename T> struct IsPairTile { static constexpr bool value = false; };
template <int NC, int TY, int H> struct IsPairTile<PairTile<NC, TY, H>> { static constexpr bool value = true; };

// Lane access to a shared tile at tile position (cx, cy): lane k of the value sits at column
// cx + k ds of a one-node tile; a pair tile holds both lanes in one slot.
template <typename V, typename T>
__device__ __forceinline__ V tld(const T& f, int i, int cy, int cx, int ds) {
    if constexpr (IsPairTile<T>::value) {
        return f.v[i][cy][cx];
    } else if constexpr (LaneTraits<V>::n == 1) {
        return f.v[i][cy][cx];
    } else {
        return make_float2(f.v[i][cy][cx], f.v[i][cy][cx + ds]);
    }
}
template <typename V, typename T>
__device__ __forceinline__ void tst(T& f, int i, int cy, int cx, int ds, V v) {
    if constexpr (IsPairTile<T>::value) {
        f.v[i][cy][cx] = v;
    } else if constexpr (LaneTraits<V>::n == 1) {
        f.v[i][cy][cx] = v;
    } else {
        f.v[i][cy][cx] = v.x;
        f.v[i][cy][cx + ds] = v.y;
    }
}

// Finite differences at tile position (cx, cy) of a field tile f (any halo >= 1).
// stencil 1 = central (Eqs. eq1stder, eq2ndder); 0 = isotropic D2Q9 stencils.
template <typename V, typename T>
__device__ __forceinline__ void grad_at(const T& f, int i, int cx, int cy, int ds, int stencil, V& gx, V& gy) {
    using E = LaneE<V>;
    const V e = tld<V>(f, i, cy, cx + 1, ds), w = tld<V>(f, i, cy, cx - 1, ds);
    const V n = tld<V>(f, i, cy + 1, cx, ds), s = tld<V>(f, i, cy - 1, cx, ds);
    if (stencil == 1) {
        gx = vmul(vbc<V>(E(0.5)), vsub(e, w));
        gy = vmul(vbc<V>(E(0.5)), vsub(n, s));
    } else {
        const V ne = tld<V>(f, i, cy + 1, cx + 1, ds), nw = tld<V>(f, i, cy + 1, cx - 1, ds);
        const V sw = tld<V>(f, i, cy - 1, cx - 1, ds), se = tld<V>(f, i, cy - 1, cx + 1, ds);
        // 3 sum_a w_a e_a h(r + e_a): 1/3 for the axis neighbours, 1/12 for the diagonals
        const V third = vbc<V>(E(1.0 / 3.0)), twelfth = vbc<V>(E(1.0 / 12.0));
        gx = vfma(vsub(e, w), third, vmul(vadd(vsub(ne, nw), vsub(se, sw)), twelfth));
        gy = vfma(vsub(n, s), third, vmul(vsub(vadd(ne, nw), vadd(sw, se)), twelfth));
    }
}

template <typename V, typename T>
__device__ __forceinline__ V lap_at(const T& f, int i, int cx, int cy, int ds, int stencil) {
    using E = LaneE<V>;
    const V c = tld<V>(f, i, cy, cx, ds);
    const V ax = vadd(vadd(tld<V>(f, i, cy, cx + 1, ds), tld<V>(f, i, cy, cx - 1, ds)),
                      vadd(tld<V>(f, i, cy + 1, cx, ds), tld<V>(f, i, cy - 1, cx, ds)));
    const V m4 = vbc<V>(E(-4));
    if (stencil == 1) return vfma(m4, c, ax);
    const V dg = vadd(vadd(tld<V>(f, i, cy + 1, cx + 1, ds), tld<V>(f, i, cy + 1, cx - 1, ds)),
                      vadd(tld<V>(f, i, cy - 1, cx - 1, ds), tld<V>(f, i, cy - 1, cx + 1, ds)));
    // 6 sum_a w_a (h(r+e_a) - h(r)): 2/3 for axis neighbours, 1/6 for diagonals
    return vfma(vfma(m4, c, ax), vbc<V>(E(2.0 / 3.0)), vmul(vfma(m4, c, dg), vbc<V>(E(1.0 / 6.0))));
}

// Sum of the nine pulled values of one component, in direction order (the order every
// kernel uses for the density of step 1, and the diagnostics for their sums).
template <typename V>
__device__ __forceinline__ V sum9(const V (&h)[9]) {
    V r = h[0];
#pragma unroll
    for (int a = 1; a < 9; ++a) r = vadd(r, h[a]);
    return r;
}

// First moment sum_i sum_a g_{a,i} e_a of the pulled values (step 1), e_a in {0, +-1}
// written out (no multiplications by zero); components in order.
template <typename V>
__device__ __forceinline__ void moment_j(const V (&h)[9], bool first, V& jx, V& jy) {
    const V jxi = vsub(vadd(vadd(h[1], h[5]), h[8]), vadd(vadd(h[3], h[6]), h[7]));
    const V jyi = vsub(vadd(vadd(h[2], h[5]), h[6]), vadd(vadd(h[4], h[7]), h[8]));
    jx = first ? jxi : vadd(jx, jxi);
    jy = first ? jyi : vadd(jy, jyi);
}

template <typename E, int NC, int TY>
struct StepSmem {
    Tile<E, NC, TY, 2> rt;   // rho~ on tile + 2
    Tile<E, NC, TY, 1> lf;   // ln f on tile + 1
    Tile<E, NC, TY, 1> G;    // Phi_i = sum_j kappa_ij lap rho~_j - RT ln f_i on tile + 1
    E Fl[2][TY][kTX];        // stored total force at the tile's nodes (lagged reading)
};

// Occupancy for two components in float storage (8-row tiles): the second component's
// nine pulled values wait in shared memory from the end of phase 1 to phase 3 instead of
// in registers, which lets the step fit 48 registers without spilling, i.e. five blocks
// of 256 threads per SM instead of four.  With three or four components the step spills
// at 48 registers even with values parked, and parking every value of a node was slower.
// The same step also addresses the distribution planes through the launch's plane
// pointers (Planes, load_gp / store_gp).
template <int NC, int ST, int TY>
constexpr bool kParkLast = ST != ST_F64 && !kLnf64<ST> && NC == 2 && TY == 8;
template <int NC, int ST, int TY>
constexpr size_t park_bytes() {
    return kParkLast<NC, ST, TY> ? (size_t)9 * TY * kTX * sizeof(typename StoreTraits<ST>::Real) : 0;
}

// The pulled value g_a of component i at this thread's node: from the parked copy
// (park[a][thread]) for the last component when the step parks it.
template <int NC, int TY, bool PARK, typename Real>
__device__ __forceinline__ void pulled_all(const Real (&g)[NC][9], const Real* park, int i, int tid, Real (&h)[9]) {
    if constexpr (PARK) {
        if (i == NC - 1) {
            const float4 a = reinterpret_cast<const float4*>(park)[tid];
            const float4 b = reinterpret_cast<const float4*>(park)[kTX * TY + tid];
            h[0] = a.x; h[1] = a.y; h[2] = a.z; h[3] = a.w;
            h[4] = b.x; h[5] = b.y; h[6] = b.z; h[7] = b.w;
            h[8] = park[8 * kTX * TY + tid];
            return;
        }
    }
#pragma unroll
    for (int a = 0; a < 9; ++a) h[a] = g[i][a];
}
template <int TY, typename Real>
__device__ __forceinline__ void park_store(const Real (&v)[9], Real* park, int tid) {
    reinterpret_cast<float4*>(park)[tid] = make_float4(v[0], v[1], v[2], v[3]);
    reinterpret_cast<float4*>(park)[kTX * TY + tid] = make_float4(v[4], v[5], v[6], v[7]);
    park[8 * kTX * TY + tid] = v[8];
}

// The stored force F(t - 1) that the lagged reading puts into u (step 1) is needed only in
// phase 3; its copy into shared memory starts before phase 1 (cp.async, no registers held)
// so that its latency hides behind phases 1 and 2 instead of stalling every warp in phase 3.
// Each thread copies and later reads only its own node's two entries.
template <typename E>
__device__ __forceinline__ void cp_async_elem(E* dst_smem, const E* src) {
    static_assert(sizeof(E) == 4 || sizeof(E) == 8, "cp.async of 4 or 8 bytes");
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    if constexpr (sizeof(E) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}

template <typename Real, int NC, int TY>
__device__ __forceinline__ void prefetch_force(const StepArgs& A, StepSmem<Real, NC, TY>& S, int tx, int ty, int gxn,
                                               int gyn, int lagged = -1) {
    if ((lagged >= 0 ? lagged != 0 : A.lagged != 0) && gxn < A.nx && gyn < A.ny) {
        const size_t nxy = (size_t)A.nx * A.ny, node = (size_t)gyn * A.nx + gxn;
        const Real* Fin = static_cast<const Real*>(A.Fin);
        cp_async_elem(&S.Fl[0][ty][tx], Fin + node);
        cp_async_elem(&S.Fl[1][ty][tx], Fin + nxy + node);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// Pull offsets: g_a(r, t) = g*_a(r - e_a, t - 1).
__device__ __forceinline__ int pull_src(int a, int wx, int wy, int xm, int xp, int ym, int yp, int nx) {
    const int sx = ex(a) == 1 ? xm : (ex(a) == -1 ? xp : wx);
    const int sy = ey(a) == 1 ? ym : (ey(a) == -1 ? yp : wy);
    return sy * nx + sx;
}

// Sum of the pulled distributions of component i at node (wx, wy) (wrapped coordinates),
// in direction order (sum9).
template <int NC, int ST, bool PP = false, bool CG = false>
__device__ __forceinline__ void pull_rho(const StepArgs& A, int wx, int wy, bool inner, int nx, int ny, int nxy,
                                         typename StoreTraits<ST>::Real* rs, const Planes* P = nullptr) {
    const int node = wy * nx + wx;
    int xm = wx - 1, xp = wx + 1, ym = wy - 1, yp = wy + 1;
    if (!inner) {
        xm = wx == 0 ? nx - 1 : xm;
        xp = wx == nx - 1 ? 0 : xp;
        ym = wy == 0 ? ny - 1 : ym;
        yp = wy == ny - 1 ? 0 : yp;
    }
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        const int src = inner ? node - ey(a) * nx - ex(a) : pull_src(a, wx, wy, xm, xp, ym, yp, nx);
#pragma unroll
        for (int i = 0; i < NC; ++i) {
            const auto v = PP ? load_gp<ST, CG>(*P, i, a, src) : load_g<ST>(A, i, a, (size_t)src, (size_t)nxy);
            rs[i] = a == 0 ? v : vadd(rs[i], v);
        }
    }
}

// Latch the first node that left the EOS domain (rho~_i <= 0, beta >= 1, non-finite ln f).
// Lane k is the node (x + k dx, y); valid_mask bit k says whether it lies in the lattice.
template <int NC, typename V>
__device__ __forceinline__ void domain_check(const StepArgs& A, const V* rt, const V* lnf, V beta, int x, int dx,
                                             int y, unsigned valid_mask) {
    using E = LaneE<V>;
#pragma unroll
    for (int k = 0; k < LaneTraits<V>::n; ++k) {
        if (!((valid_mask >> k) & 1u)) continue;
        bool bad = !(lane(beta, k) < E(1));
        int badc = 0;
#pragma unroll
        for (int i = NC - 1; i >= 0; --i) {
            if (!(lane(rt[i], k) > E(0)) || !isfinite(lane(lnf[i], k))) {
                badc = i;
                bad = true;
            }
        }
        // a plain read first: once a lattice has failed, every bad node would otherwise
        // contend for the same word with an atomic in every step
        if (bad && *reinterpret_cast<volatile int*>(&A.err->flag) == 0 && atomicCAS(&A.err->flag, 0, 1) == 0) {
            A.err->comp = badc;
            A.err->x = x + k * dx;
            A.err->y = y;
        }
    }
}

// ---- the phases of one tile, shared by every variant of the step kernel (so all variants
//      perform the same arithmetic in the same order and agree bit for bit) ----

// Phase 1, the node owned by this thread: rho_i and the first moment (step 1, returned in
// r, jx, jy) and rho~, ln f (steps 2-5) from its nine pulled values per component.
template <int NC, int TY, typename Real, bool LNF64 = false>
__device__ __forceinline__ void phase1_node(const StepArgs& A, const MixConstT<Real>& m, StepSmem<Real, NC, TY>& S,
                                            const Real (&g)[NC][9], Real (&r)[NC], Real& jx, Real& jy, int tx, int ty,
                                            bool valid, int gx, int gy, int eos = -1) {
    Real rt[NC], lnf[NC];
#pragma unroll
    for (int i = 0; i < NC; ++i) {
        r[i] = sum9(g[i]);
        moment_j(g[i], i == 0, jx, jy);
        rt[i] = vmul(r[i], m.invM[i]);
        S.rt.v[i][ty + 2][tx + 2] = rt[i];
    }
    const Real beta = node_lnf_st<NC, LNF64, Real>(A, m, rt, lnf, eos);
#pragma unroll
    for (int i = 0; i < NC; ++i) S.lf.v[i][ty + 1][tx + 1] = lnf[i];
    domain_check<NC, Real>(A, rt, lnf, beta, gx, 0, gy, valid && checked_row(A, gy) ? 1u : 0u);
}

// Ring position r (0 <= r < 4 (TW + 4) + 4 TY) -> box coordinates (bx, by) of the 2-node halo
// ring around a TW x TY tile (box origin at tile origin - (2, 2)), row by row.  (Putting the
// inner-ring positions, which also need ln f, first measured slower.)
template <int TY, int TW = kTX>
__device__ __forceinline__ void ring_position(int r, int& bx, int& by) {
    constexpr int WB = TW + 4;
    if (r < 2 * WB) {
        by = r / WB;
        bx = r % WB;
    } else if (r < 4 * WB) {
        by = TY + 2 + (r - 2 * WB) / WB;
        bx = (r - 2 * WB) % WB;
    } else {
        const int q = r - 4 * WB;
        by = 2 + (q >> 2);
        const int c = q & 3;
        bx = c < 2 ? c : TW + c;  // 0, 1, TW+2, TW+3
    }
}

// Phase 1, a halo ring node: rho~ from its summed densities; ln f on the inner 1-node ring.
template <int NC, int TY, typename Real, bool LNF64 = false>
__device__ __forceinline__ void phase1_ring(const StepArgs& A, const MixConstT<Real>& m, StepSmem<Real, NC, TY>& S,
                                            Real (&rt)[NC], int bx, int by, int eos = -1) {
#pragma unroll
    for (int i = 0; i < NC; ++i) {
        rt[i] = vmul(rt[i], m.invM[i]);
        S.rt.v[i][by][bx] = rt[i];
    }
    if (bx >= 1 && bx <= kTX + 2 && by >= 1 && by <= TY + 2) {
        Real lnf[NC];
        node_lnf_st<NC, LNF64, Real>(A, m, rt, lnf, eos);
#pragma unroll
        for (int i = 0; i < NC; ++i) S.lf.v[i][by - 1][bx - 1] = lnf[i];
    }
}

// Phase 2 at box position (cx, cy) of the tile + 1 box (lane k at cx + k ds):
// G_i = sum_j kappa_ij lap rho~_j (step 6, mu_I,i = -G_i), stored as the potential
// Phi_i = G_i - RT ln f_i whose gradient times rho~_i is the force of step 7.
template <int NC, typename V, typename E, typename TR, typename TL, typename TG>
__device__ __forceinline__ void phase2_core(const MixConstT<E>& m, const TR& rt, const TL& lf, TG& G, int stencil,
                                            int cx, int cy, int ds) {
    V L[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) L[j] = lap_at<V>(rt, j, cx + 1, cy + 1, ds, stencil);
    const V mRT = vbc<V>(-m.RT);
#pragma unroll
    for (int i = 0; i < NC; ++i) {
        V Gi = vmul(vbc<V>(m.kap[i * kMaxC]), L[0]);
#pragma unroll
        for (int j = 1; j < NC; ++j) Gi = vfma(vbc<V>(m.kap[i * kMaxC + j]), L[j], Gi);
        tst<V>(G, i, cy, cx, ds, vfma(mRT, tld<V>(lf, i, cy, cx, ds), Gi));
    }
}

// The tile + 1 box has TY + 2 rows of 32 + 2 columns.  Each warp takes whole rows of the
// first 32 columns (one shared-memory row per instruction: no bank conflicts, no index
// division); the last warp, which has one row, also takes the two edge columns.
template <int NC, int TY, typename Real>
__device__ __forceinline__ void phase2(const MixConstT<Real>& m, StepSmem<Real, NC, TY>& S, int stencil, int tid) {
    const int tx = tid & (kTX - 1), ty = tid / kTX;
    for (int cy = ty; cy < TY + 2; cy += TY) phase2_core<NC, Real>(m, S.rt, S.lf, S.G, stencil, tx, cy, 0);
    if (ty == TY - 1)
        for (int e = tx; e < 2 * (TY + 2); e += kTX)
            phase2_core<NC, Real>(m, S.rt, S.lf, S.G, stencil, kTX + (e & 1), e >> 1, 0);
}

// Phase 3 at one lane of nodes: force (step 7), velocity (step 1), equilibrium and
// forcing (step 8) and collision (step 9).
//   Gt, Rt: the Phi tile (tile + 1) and the rho~ tile (tile + 2); (cx, cy) the node's
//           position in the tile + 1 coordinates, lane k at cx + k ds;
//   rho, jx, jy: the component densities and the total first moment of step 1 (phase 1);
//   geth(i, h): the nine pulled values of component i;
//   Fpx, Fpy: the stored total force F(t - 1) (LAG: the lagged reading; ignored otherwise);
//   COLLIDE = false: velocity only (macroscopic fields); else store(i, a, value) receives
//           every post-collision value; Ft is the total force of this step.
// Under the lagged reading u is known before any force of this step, so each component's
// force goes straight into its collision (no per-component arrays held in registers).
// STD: the standard formulation of Section VI -- equilibrium rho_i w_a [1 + ...] of
// Eq. eqLBE, Guo's forcing term of Eq. eqLBEfinal3 (no grad rho_i part) and
// F_i + c_s^2 grad rho_i of Eq. eqForceGen.
template <int NC, bool COLLIDE, bool STD, bool LAG, typename V, typename E, typename TG, typename TR, typename GetH,
          typename Store>
__device__ __forceinline__ void phase3_core(const MixConstT<E>& m, int stencil, const TG& Gt, const TR& Rt, int cx,
                                            int cy, int ds, const V (&rho)[NC], V jx, V jy, GetH&& geth, V Fpx,
                                            V Fpy, Store&& store, V& Ftx, V& Fty, V& ux, V& uy) {
    // F_i and grad rho_i of component i
    auto force = [&](int i, V& Fx, V& Fy, V& grx, V& gry) {
        V px, py, rx, ry;
        grad_at<V>(Gt, i, cx, cy, ds, stencil, px, py);
        grad_at<V>(Rt, i, cx + 1, cy + 1, ds, stencil, rx, ry);
        const V rti = tld<V>(Rt, i, cy + 1, cx + 1, ds);
        // grad rho_i = M_i grad rho~_i
        grx = vmul(rx, vbc<V>(m.M[i]));
        gry = vmul(ry, vbc<V>(m.M[i]));
        // Eq. eqforcefinal: F_i = -rho~_i RT grad ln f_i + rho~_i grad(sum_j kappa_ij lap rho~_j)
        //                      = rho~_i grad Phi_i (the stencils are linear)
        Fx = vmul(rti, px);
        Fy = vmul(rti, py);
        if constexpr (STD) {  // Eq. eqForceGen: + c_s^2 grad rho_i
            Fx = vfma(vbc<V>(E(1.0 / 3.0)), grx, Fx);
            Fy = vfma(vbc<V>(E(1.0 / 3.0)), gry, Fy);
        }
        Ftx = i == 0 ? Fx : vadd(Ftx, Fx);
        Fty = i == 0 ? Fy : vadd(Fty, Fy);
    };
    V rho_t = rho[0];
#pragma unroll
    for (int i = 1; i < NC; ++i) rho_t = vadd(rho_t, rho[i]);
    const V half = vbc<V>(E(0.5));
    const V inv_rho = vrcp(rho_t);
    // Collision g' = g - omega (g - g^eq) + fcoef F_a, with g^eq of Eq. eqLBEMCb (rho_0 = 0)
    // and F_a of Eq. eqLBEMCfinal3, evaluated for each pair of opposite directions
    // (e_abar = -e_a): the parts even in e are shared, the odd parts change sign.
    //   g^eq_a = w rho [3 eu + 4.5 eu^2 - 1.5 u^2]
    //   F_a    = w [3 eF - 3 uF + 9 eu eF + (c_a - 1) ug + 3 eu eg],  c_a = (3 e^2 - 2)/2
    // (eu = e_a.u, eF = e_a.F_i, eg = e_a.grad rho_i, uF = u.F_i, ug = u.grad rho_i).  With
    // rw = omega rho_i, fc = fcoef, base = 1.5 rw u^2 the post-collision value is
    //   g'_a = (1 - omega) g_a + even_a + odd_a,   g'_abar = (1 - omega) g_abar + even_a - odd_a
    //   even_a = w_a [eu (e_a.V) + cb_a],  V = 4.5 rw u + fc (9 F_i + 3 grad rho_i),
    //            cb_a = fc (c_a - 1) ug - 3 fc uF - base
    //   odd_a  = 3 w_a (rw eu + fc eF) = e_a.O (axes), e_a.O / 4 (diagonals),
    //            O = (rw u + fc F_i) / 3
    //   g'_0   = (1 - omega) g_0 + rw + (4/9) (-base - 3 fc uF - 2 fc ug)
    // and each e_a.X is written out (components 0, +-1): no multiplication by zero.
    auto collide = [&](int i, V Fx, V Fy, V grx, V gry) {
        const E fc = m.fcoef;
        const V usq15 = vmul(vbc<V>(E(1.5)), vfma(ux, ux, vmul(uy, uy)));
        V h[9];
        geth(i, h);
        const V rw = vmul(vbc<V>(m.omega), rho[i]);
        const V uF = vfma(ux, Fx, vmul(uy, Fy));
        const V a0 = vneg(vfma(rw, usq15, vmul(vbc<V>(E(3) * fc), uF)));  // -base - 3 fc uF
        V cb_ax, cb_dg, Vx, Vy, g0c;
        if constexpr (STD) {
            // the forcing term's grad rho_i part belongs to the well-balanced scheme only;
            // the standard equilibrium adds w_a rho_i (a != 0) and w_0 rho_i (a = 0)
            cb_ax = vadd(a0, rw);
            cb_dg = cb_ax;
            Vx = vfma(vbc<V>(E(4.5)), vmul(rw, ux), vmul(vbc<V>(E(9) * fc), Fx));
            Vy = vfma(vbc<V>(E(4.5)), vmul(rw, uy), vmul(vbc<V>(E(9) * fc), Fy));
            g0c = vmul(vbc<V>(E(4.0 / 9.0)), vadd(rw, a0));
        } else {
            const V ug = vfma(ux, grx, vmul(uy, gry));
            cb_ax = vfma(vbc<V>(E(-0.5) * fc), ug, a0);
            cb_dg = vfma(vbc<V>(fc), ug, a0);
            Vx = vfma(vbc<V>(E(4.5)), vmul(rw, ux), vfma(vbc<V>(E(9) * fc), Fx, vmul(vbc<V>(E(3) * fc), grx)));
            Vy = vfma(vbc<V>(E(4.5)), vmul(rw, uy), vfma(vbc<V>(E(9) * fc), Fy, vmul(vbc<V>(E(3) * fc), gry)));
            g0c = vfma(vbc<V>(E(4.0 / 9.0)), vfma(vbc<V>(E(-2) * fc), ug, a0), rw);
        }
        const V rw3 = vmul(rw, vbc<V>(E(1.0 / 3.0)));
        const V fc_3 = vbc<V>(fc * E(1.0 / 3.0));
        const V Ox = vfma(rw3, ux, vmul(fc_3, Fx));
        const V Oy = vfma(rw3, uy, vmul(fc_3, Fy));
        const V keep = vbc<V>(E(1) - m.omega);
        const V w1 = vbc<V>(E(1.0 / 9.0)), w5 = vbc<V>(E(1.0 / 36.0)), quarter = vbc<V>(E(0.25));
        // g'_a = keep g_a + (w_a X_a +- odd_a), X_a = eu (e_a.V) + cb_a: one fused product each
        store(i, 0, vfma(keep, h[0], g0c));
        const V X1 = vfma(ux, Vx, cb_ax);
        store(i, 1, vfma(keep, h[1], vfma(w1, X1, Ox)));
        store(i, 3, vfma(keep, h[3], vfma(w1, X1, vneg(Ox))));
        const V X2 = vfma(uy, Vy, cb_ax);
        store(i, 2, vfma(keep, h[2], vfma(w1, X2, Oy)));
        store(i, 4, vfma(keep, h[4], vfma(w1, X2, vneg(Oy))));
        const V X5 = vfma(vadd(ux, uy), vadd(Vx, Vy), cb_dg), o5 = vmul(quarter, vadd(Ox, Oy));
        store(i, 5, vfma(keep, h[5], vfma(w5, X5, o5)));
        store(i, 7, vfma(keep, h[7], vfma(w5, X5, vneg(o5))));
        const V X6 = vfma(vsub(uy, ux), vsub(Vy, Vx), cb_dg), o6 = vmul(quarter, vsub(Oy, Ox));
        store(i, 6, vfma(keep, h[6], vfma(w5, X6, o6)));
        store(i, 8, vfma(keep, h[8], vfma(w5, X6, vneg(o6))));
    };
    if constexpr (LAG) {
        ux = vmul(vfma(half, Fpx, jx), inv_rho);
        uy = vmul(vfma(half, Fpy, jy), inv_rho);
#pragma unroll
        for (int i = 0; i < NC; ++i) {
            V Fx, Fy, grx, gry;
            force(i, Fx, Fy, grx, gry);
            if constexpr (COLLIDE) collide(i, Fx, Fy, grx, gry);
        }
    } else {
        V Fx[NC], Fy[NC], grx[NC], gry[NC];
#pragma unroll
        for (int i = 0; i < NC; ++i) force(i, Fx[i], Fy[i], grx[i], gry[i]);
        ux = vmul(vfma(half, Ftx, jx), inv_rho);
        uy = vmul(vfma(half, Fty, jy), inv_rho);
        if constexpr (COLLIDE) {
#pragma unroll
            for (int i = 0; i < NC; ++i) collide(i, Fx[i], Fy[i], grx[i], gry[i]);
        }
    }
}

// Phase 3 of the one-node-per-thread kernels at one valid node.
template <int NC, int ST, int TY, bool MOMENTS, bool STD = false, bool PARK = false, bool PP = false>
__device__ __forceinline__ void phase3(const StepArgs& A, const MixConstT<typename StoreTraits<ST>::Real>& m,
                                       StepSmem<typename StoreTraits<ST>::Real, NC, TY>& S,
                                       const typename StoreTraits<ST>::Real (&g)[NC][9],
                                       const typename StoreTraits<ST>::Real (&rho)[NC],
                                       typename StoreTraits<ST>::Real jx, typename StoreTraits<ST>::Real jy, int tx,
                                       int ty, int gxn, int gyn, const typename StoreTraits<ST>::Real* park = nullptr,
                                       const Planes* P = nullptr, int stencil = -1, int lagged = -1) {
    using Real = typename StoreTraits<ST>::Real;
    const int nx = A.nx, nxy = A.nx * A.ny;
    const int node = gyn * nx + gxn;
    const int tid = ty * kTX + tx;
    auto geth = [&](int i, Real (&h)[9]) { pulled_all<NC, TY, PARK, Real>(g, park, i, tid, h); };
    auto store = [&](int i, int a, Real v) { store_gsel<ST, PP>(A, P, i, a, node, nxy, v); };
    Real Ftx, Fty, ux, uy;
    const int sten = stencil >= 0 ? stencil : A.stencil;
    if (lagged >= 0 ? lagged != 0 : A.lagged != 0) {  // F(t - 1), copied by prefetch_force
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        const Real Fpx = S.Fl[0][ty][tx], Fpy = S.Fl[1][ty][tx];
        phase3_core<NC, !MOMENTS, STD, true, Real>(m, sten, S.G, S.rt, tx + 1, ty + 1, 0, rho, jx, jy, geth, Fpx,
                                                   Fpy, store, Ftx, Fty, ux, uy);
    } else {
        phase3_core<NC, !MOMENTS, STD, false, Real>(m, sten, S.G, S.rt, tx + 1, ty + 1, 0, rho, jx, jy, geth,
                                                    Real(0), Real(0), store, Ftx, Fty, ux, uy);
    }
    if constexpr (MOMENTS) {
#pragma unroll
        for (int i = 0; i < NC; ++i) {
            if (A.rho_out) A.rho_out[(size_t)i * nxy + node] = (double)rho[i];
            if (A.lnf_out) A.lnf_out[(size_t)i * nxy + node] = (double)S.lf.v[i][ty + 1][tx + 1];
        }
        if (A.u_out) {
            A.u_out[node] = (double)ux;
            A.u_out[(size_t)nxy + node] = (double)uy;
        }
    } else {
        Real* Fout = static_cast<Real*>(A.Fout);
        Fout[node] = Ftx;
        Fout[nxy + node] = Fty;
    }
}

// Phase 1 from global memory for one tile: pull of the owned node (into g, its densities
// into r) and of the halo ring (rho~ only), with periodic wrap unless the tile is inner.
// INNER = 1 / 0: the tile is / is not inner, known where the code is compiled (a separate code
// path for the wrap-free tiles); -1: the argument says.
template <int NC, int ST, int TY, bool PP = false, int INNER = -1, bool CG = false>
__device__ __forceinline__ void phase1_global(const StepArgs& A, const MixConstT<typename StoreTraits<ST>::Real>& m,
                                              StepSmem<typename StoreTraits<ST>::Real, NC, TY>& S,
                                              typename StoreTraits<ST>::Real (&g)[NC][9],
                                              typename StoreTraits<ST>::Real (&r)[NC],
                                              typename StoreTraits<ST>::Real& jx, typename StoreTraits<ST>::Real& jy,
                                              int x0, int y0, bool inner_arg, int tx, int ty, int tid,
                                              const Planes* P = nullptr, int eos = -1) {
    const bool inner = INNER >= 0 ? INNER == 1 : inner_arg;
    using Real = typename StoreTraits<ST>::Real;
    constexpr int NT = kTX * TY;
    const int nx = A.nx, ny = A.ny, nxy = nx * ny;
    const int gxn = x0 + tx, gyn = y0 + ty;
    const bool valid = gxn < nx && gyn < ny;
    // Each thread owns one node and at most one ring node.  Ring first (measured faster
    // except for three or four components in FP32, where it holds too many registers): the
    // ring node's pulled sums arrive, then the owned node's loads are issued and the ring
    // node's ln f is computed while they are in flight.  Otherwise the owned node comes
    // first and the ring node after it.
    constexpr int RING = 4 * (kTX + 4) + 4 * TY;
    static_assert(RING <= NT, "one ring node per thread");
    constexpr bool RING_FIRST = !(ST == ST_F32 && NC >= 3);
    const bool has_ring = tid < RING;
    int bx = 0, by = 0;
    Real rr[NC];
    auto pull_ring = [&]() {
        ring_position<TY>(tid, bx, by);
        const int wx = inner ? x0 - 2 + bx : wrap(x0 - 2 + bx, nx);
        const int wy = inner ? y0 - 2 + by : wrap(y0 - 2 + by, ny);
        pull_rho<NC, ST, PP, CG>(A, wx, wy, inner, nx, ny, nxy, rr, P);
    };
    if (RING_FIRST && has_ring) pull_ring();
    {
        const int wx = inner ? gxn : wrap(gxn, nx), wy = inner ? gyn : wrap(gyn, ny);
        const int node = wy * nx + wx;
        int xm = wx - 1, xp = wx + 1, ym = wy - 1, yp = wy + 1;
        if (!inner) {
            xm = wx == 0 ? nx - 1 : xm;
            xp = wx == nx - 1 ? 0 : xp;
            ym = wy == 0 ? ny - 1 : ym;
            yp = wy == ny - 1 ? 0 : yp;
        }
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            const int src = inner ? node - ey(a) * nx - ex(a) : pull_src(a, wx, wy, xm, xp, ym, yp, nx);
#pragma unroll
            for (int i = 0; i < NC; ++i)
                g[i][a] = PP ? load_gp<ST, CG>(*P, i, a, src) : load_g<ST>(A, i, a, (size_t)src, (size_t)nxy);
        }
    }
    if constexpr (RING_FIRST) {
        if (has_ring) phase1_ring<NC, TY, Real, kLnf64<ST>>(A, m, S, rr, bx, by, eos);
        phase1_node<NC, TY, Real, kLnf64<ST>>(A, m, S, g, r, jx, jy, tx, ty, valid, gxn, gyn, eos);
    } else {
        phase1_node<NC, TY, Real, kLnf64<ST>>(A, m, S, g, r, jx, jy, tx, ty, valid, gxn, gyn, eos);
        if (has_ring) {
            pull_ring();
            phase1_ring<NC, TY, Real, kLnf64<ST>>(A, m, S, rr, bx, by, eos);
        }
    }
}

// ---- compensated sums of the diagnostics ----
// The masses and residual sums are accumulated in double precision from the strip level up
// (8 warp rows of 32 nodes).  Below that, in a warp, a float lane carries each sum as an
// unevaluated pair hi + lo of floats (float-float, about 44 significant bits) built from exact
// sums and products, which costs a few FP32 instructions per node instead of FP64 ones (GB300
// executes about 2 FP64 operations per clock per SM, 1/64 of its FP32 rate).  Double lanes (the
// FP64 storage) sum in plain double, lo staying 0.
template <typename V>
struct Sum2 {
    V hi, lo;
};
template <typename V> constexpr bool kCompensated = !std::is_same<LaneE<V>, double>::value;

template <typename V>
__device__ __forceinline__ Sum2<V> s2_of(V a) { return {a, vbc<V>(LaneE<V>(0))}; }
// s + e = a + b exactly (Knuth's two-sum)
template <typename V>
__device__ __forceinline__ Sum2<V> two_sum(V a, V b) {
    if constexpr (!kCompensated<V>) {
        return s2_of(vadd(a, b));
    } else {
        const V s = vadd(a, b), bb = vsub(s, a);
        return {s, vadd(vsub(a, vsub(s, bb)), vsub(b, bb))};
    }
}
// p + e = a b exactly (the rounding error of a product is a fused multiply-add away)
template <typename V>
__device__ __forceinline__ Sum2<V> two_prod(V a, V b) {
    const V p = vmul(a, b);
    if constexpr (!kCompensated<V>) return s2_of(p);
    else return {p, vfma(a, b, vneg(p))};
}
// (a.hi + a.lo) + (b.hi + b.lo), renormalised so that |lo| <= ulp(hi) / 2
template <typename V>
__device__ __forceinline__ Sum2<V> s2_add(Sum2<V> a, Sum2<V> b) {
    if constexpr (!kCompensated<V>) {
        return s2_of(vadd(a.hi, b.hi));
    } else {
        const Sum2<V> t = two_sum(a.hi, b.hi);
        const V e = vadd(t.lo, vadd(a.lo, b.lo));
        const V hi = vadd(t.hi, e);
        return {hi, vsub(e, vsub(hi, t.hi))};
    }
}

// Diagnostics sums at one node (lane), shared by reduce_partial and the fused steps so that
// all give the same bits: rho_i, (rho_i - pv_i)^2 (0 without a snapshot) and rho_i^2 into
// acc.  The callers read the snapshot pv whatever have_prev says (its buffer always holds
// N x nx x ny values) and early: a read guarded by the flag was issued only after the
// pulled sums had arrived and made the reduction about three times slower.
template <int NC, typename V>
__device__ __forceinline__ void diag_node(const V (&r)[NC], const V (&pv)[NC], int have_prev, Sum2<V> (&acc)[NC + 2]) {
#pragma unroll
    for (int i = 0; i < NC; ++i) {
        acc[i] = s2_of(r[i]);
        const Sum2<V> sq = two_prod(r[i], r[i]);
        acc[NC + 1] = i == 0 ? sq : s2_add(acc[NC + 1], sq);
        Sum2<V> d2 = s2_of(vbc<V>(LaneE<V>(0)));
        if (have_prev) {
            // d = r - pv exactly as dh + dl; d^2 = dh^2 + 2 dh dl to the working precision
            const Sum2<V> d = two_sum(r[i], vneg(pv[i]));
            d2 = two_prod(d.hi, d.hi);
            if constexpr (kCompensated<V>) d2.lo = vfma(vadd(d.hi, d.hi), d.lo, d2.lo);
        }
        acc[NC] = i == 0 ? d2 : s2_add(acc[NC], d2);
    }
}

__device__ __forceinline__ float shfl_xor(float v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double shfl_xor(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ float2 shfl_xor(float2 v, int o) {
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
}
template <typename V>
__device__ __forceinline__ Sum2<V> shfl_xor(const Sum2<V>& v, int o) {
    Sum2<V> w;
    w.hi = shfl_xor(v.hi, o);
    w.lo = kCompensated<V> ? shfl_xor(v.lo, o) : v.lo;
    return w;
}

// Warp sums of K compensated sums into one row of a per-block table (a fixed order, so every
// kernel that reduces the same nodes gets the same bits).  A transposed reduction: with the K
// sums padded to a power of two KP, at each of the first log2 KP levels (lane distances 16, 8,
// ...) a lane keeps half of its sums, receives its partner's copies of them and adds them, and
// passes the other half to the partner, so each pair-sum is formed once; then each group of
// 32 / KP lanes holds one sum and finishes it with a butterfly.  About 2 KP adds per lane in
// all, where a butterfly per sum takes 5 levels for each of the K sums.
constexpr int pow2_at_least(int k) { return k <= 1 ? 1 : 2 * pow2_at_least((k + 1) / 2); }
template <int K, typename V>
__device__ __forceinline__ void sums_warp(const Sum2<V> (&acc)[K], Sum2<V>* row) {
    static_assert(K >= 1 && K <= 32, "up to 32 sums per warp");
    constexpr int KP = pow2_at_least(K);
    const int lane = threadIdx.x & 31;
    Sum2<V> v[KP];
#pragma unroll
    for (int j = 0; j < KP; ++j) v[j] = j < K ? acc[j] : s2_of(vbc<V>(LaneE<V>(0)));
    int q = 0;  // index of the first sum this lane still holds
#pragma unroll
    for (int h = KP / 2, o = 16; h >= 1; h >>= 1, o >>= 1) {
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int j = 0; j < h; ++j) {
            const Sum2<V> keep = upper ? v[j + h] : v[j];
            const Sum2<V> send = upper ? v[j] : v[j + h];
            v[j] = s2_add(keep, shfl_xor(send, o));
        }
        q += upper ? h : 0;
    }
#pragma unroll
    for (int o = 16 / KP; o >= 1; o >>= 1) v[0] = s2_add(v[0], shfl_xor(v[0], o));
    if ((lane & (32 / KP - 1)) == 0 && q < K) row[q] = v[0];
}
template <int NC, typename V>
__device__ __forceinline__ void diag_warp(const Sum2<V> (&acc)[NC + 2], Sum2<V>* row) {
    sums_warp<NC + 2, V>(acc, row);
}

// Sum in double of eight consecutive rows of that table, in row order (one 32 x 8 strip), for
// lane l of the lane type.
template <int K, typename V>
__device__ __forceinline__ double sums_strip(const Sum2<V> (*red)[K], int row0, int k, int l) {
    double v = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        v += (double)lane(red[row0 + w][k].hi, l);
        if constexpr (kCompensated<V>) v += (double)lane(red[row0 + w][k].lo, l);
    }
    return v;
}
template <int NC, typename V>
__device__ __forceinline__ double diag_strip(const Sum2<V> (*red)[NC + 2], int row0, int k, int l) {
    return sums_strip<NC + 2, V>(red, row0, k, l);
}

// The phase measure's node terms: ln rho_i.  A sum over a periodic lattice of a smooth
// function of the densities does not change when the density field moves rigidly (a flat
// or curved interface drifting with the momentum the transient left, which nothing damps in
// a periodic box), while it follows every change of the phases themselves: its change over
// a check interval, divided by the node count, is the volume-averaged relative change of
// rho_i.
template <int NC, typename V>
__device__ __forceinline__ void lnrho_node(const V (&r)[NC], Sum2<V> (&acc)[NC]) {
#pragma unroll
    for (int i = 0; i < NC; ++i) acc[i] = s2_of(vln(r[i]));
}

// Diagnostics of the state a step reads, fused into the step (A.diag_partial set): the
// snapshot value of each owned node is copied into shared memory before phase 1, and after
// phase 3 each 32 x 8 strip of the tile writes its N + 2 partial sums at the index
// reduce_partial would use ((strip row) * tiles_x + tile column), and the snapshot takes
// the densities of this state.
template <int NC, typename Real, int TY>
__device__ __forceinline__ void diag_prefetch(const StepArgs& A, Real* pv_s, int tx, int ty, int gxn, int gyn) {
    if (A.diag_partial != nullptr && gxn < A.nx && gyn < A.ny) {
        const Real* prev = static_cast<const Real*>(A.rho_prev);
        const size_t nxy = (size_t)A.nx * A.ny, node = (size_t)gyn * A.nx + gxn;
#pragma unroll
        for (int i = 0; i < NC; ++i) cp_async_elem(&pv_s[(i * TY + ty) * kTX + tx], prev + i * nxy + node);
    }
}

// Called by every thread of the block (it synchronises); uniform in A.diag_partial.
template <int NC, typename Real, int TY>
__device__ __forceinline__ void diag_tile(const StepArgs& A, const Real (&r)[NC], const Real* pv_s, int tx, int ty,
                                          int gxn, int gyn, int y0, int tile_row, int tile_col, int tiles_x) {
    static_assert(TY % 8 == 0, "diagnostics strips of 8 rows");
    __shared__ Sum2<Real> dred[TY][NC + 2];
    const int nx = A.nx, ny = A.ny, tid = ty * kTX + tx;
    Sum2<Real> acc[NC + 2];
#pragma unroll
    for (int k = 0; k < NC + 2; ++k) acc[k] = s2_of(Real(0));
    if (gxn < nx && gyn < ny) {
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        Real pv[NC];
#pragma unroll
        for (int i = 0; i < NC; ++i) pv[i] = pv_s[(i * TY + ty) * kTX + tx];
        diag_node<NC, Real>(r, pv, A.have_prev, acc);
        Real* prev = static_cast<Real*>(A.rho_prev);
        const size_t nxy = (size_t)nx * ny, node = (size_t)gyn * nx + gxn;
#pragma unroll
        for (int i = 0; i < NC; ++i) prev[i * nxy + node] = r[i];
    }
    diag_warp<NC, Real>(acc, dred[ty]);
    __syncthreads();
    constexpr int STRIPS = TY / 8;
    if (tid < STRIPS * (NC + 2)) {
        const int sub = tid / (NC + 2), k = tid % (NC + 2);
        if (y0 + 8 * sub < ny)
            static_cast<double*>(A.diag_partial)[((size_t)(tile_row * STRIPS + sub) * tiles_x + tile_col) * (NC + 2) + k] =
                diag_strip<NC, Real>(dred, 8 * sub, k, 0);
    }
}

// MOMENTS = true: compute the macroscopic fields of the current state instead of
// advancing it (no distribution or force store).
// SPEC = true: the instantiation for the Peng-Robinson EOS, isotropic stencils and the lagged
// velocity reading (well-balanced formulation), compiled with those choices as constants (no
// branches on them) and with separate code paths for wrap-free and edge tiles; the launcher
// picks it only for lattices with those options.  The arithmetic is the generic kernel's.
template <int NC, int ST, int TY, bool MOMENTS, bool STD = false, bool SPEC = false>
// Float arithmetic: 1024 resident threads per SM (64 registers a thread), measured faster
// than trading occupancy for registers (77 registers and three 8-row blocks per SM were 7%
// slower for three components) or registers for occupancy (48 registers spill).  More
// resident blocks did not help where they fit either: the specialised two-component step
// fits 40 registers without spilling, but six blocks per SM ran 5% slower than five (more
// warps contend for the same L1 and L2 traffic).  The FP64 reference path keeps what the
// compiler chooses.
__global__ void __launch_bounds__(kTX* TY, ST == ST_F64 ? 1 : (kParkLast<NC, ST, TY> ? 5 : 1024 / (kTX * TY)))
    fused_step(StepArgs A, Planes P) {
    using Real = typename StoreTraits<ST>::Real;
    constexpr bool PARK = kParkLast<NC, ST, TY>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto& S = *reinterpret_cast<StepSmem<Real, NC, TY>*>(smem_raw);
    // dynamic shared memory: StepSmem, the parked values (PARK), the diagnostics snapshot
    Real* park = reinterpret_cast<Real*>(smem_raw + sizeof(StepSmem<Real, NC, TY>));
    const MixConstT<Real>& m = mixc<Real>(A);
    const int nx = A.nx, ny = A.ny;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * kTX + tx;
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * TY;
    // no periodic wrap anywhere in this block's reach (tile + 2 halo + 1 pull)
    const bool inner = x0 >= 3 && x0 + kTX + 3 <= nx && y0 >= 3 && y0 + TY + 3 <= ny;
    const int gxn = x0 + tx, gyn = y0 + ty;
    // diagnostics: the density snapshot of this thread's node, copied like the force (a load
    // issued after phase 3 stalled the whole step about 2x)
    Real* pv_s = reinterpret_cast<Real*>(smem_raw + sizeof(StepSmem<Real, NC, TY>) + park_bytes<NC, ST, TY>());
    static_assert(!SPEC || (!MOMENTS && !STD), "the specialised step advances the well-balanced scheme");
    const int eos = SPEC ? 0 : -1;               // Peng-Robinson
    const int stencil = SPEC ? 0 : A.stencil;    // isotropic
    const int lagged = SPEC ? 1 : -1;
    if constexpr (!MOMENTS) diag_prefetch<NC, Real, TY>(A, pv_s, tx, ty, gxn, gyn);
    prefetch_force<Real, NC, TY>(A, S, tx, ty, gxn, gyn, lagged);
    Real g[NC][9], r[NC], jx, jy;
    if constexpr (SPEC) {
        if (inner)
            phase1_global<NC, ST, TY, PARK, 1>(A, m, S, g, r, jx, jy, x0, y0, true, tx, ty, tid, &P, eos);
        else
            phase1_global<NC, ST, TY, PARK, 0>(A, m, S, g, r, jx, jy, x0, y0, false, tx, ty, tid, &P, eos);
    } else {
        phase1_global<NC, ST, TY, PARK>(A, m, S, g, r, jx, jy, x0, y0, inner, tx, ty, tid, &P);
    }
    if constexpr (PARK) park_store<TY, Real>(g[NC - 1], park, tid);
    __syncthreads();
    phase2<NC, TY, Real>(m, S, stencil, tid);
    __syncthreads();
    if (gxn < nx && gyn < ny)
        phase3<NC, ST, TY, MOMENTS, STD, PARK, PARK>(A, m, S, g, r, jx, jy, tx, ty, gxn, gyn, park, &P, stencil,
                                                     lagged);
    if constexpr (!MOMENTS) {
        if (A.diag_partial != nullptr)  // uniform: diagnostics of the state this step read
            diag_tile<NC, Real, TY>(A, r, pv_s, tx, ty, gxn, gyn, y0, blockIdx.y, blockIdx.x, gridDim.x);
    }
}

// g = g^eq(rho, u = 0): rho_i in a = 0, zero elsewhere (well-balanced); w_a rho_i in every
// direction (standard formulation, stored where the next pull reads it); stored force zero.
template <int NC, int ST>
__global__ void init_rest(StepArgs A, const double* __restrict__ rho) {
    using Real = typename StoreTraits<ST>::Real;
    const size_t nxy = (size_t)A.nx * A.ny;
    for (size_t node = blockIdx.x * (size_t)blockDim.x + threadIdx.x; node < nxy;
         node += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int i = 0; i < NC; ++i) {
            const Real r = (Real)rho[(size_t)i * nxy + node];
            if (!A.standard) {
#pragma unroll
                for (int a = 0; a < 9; ++a) store_g<ST>(A, i, a, node, nxy, a == 0 ? r : Real(0));
            } else {
                // the buffer holds what the next pull reads: g_a(s + e_a) is stored at s, so
                // direction a takes w_a rho at the node s + e_a (periodic)
                const int x = (int)(node % A.nx), y = (int)(node / A.nx);
#pragma unroll
                for (int a = 0; a < 9; ++a) {
                    const int xs = wrap(x + ex(a), A.nx), ys = wrap(y + ey(a), A.ny);
                    const Real ra = (Real)rho[(size_t)i * nxy + (size_t)ys * A.nx + xs];
                    store_g<ST>(A, i, a, node, nxy, wgt<Real>(a) * ra);
                }
            }
        }
        Real* F = static_cast<Real*>(A.Fout);
        F[node] = Real(0);
        F[nxy + node] = Real(0);
    }
}

// Post-streaming distributions <-> storage: g_a(r) = g*_a(r - e_a).
// to_storage = true: gin_d (double, [N][9][ny][nx] post-streaming) -> storage (A.gout);
// false: storage (A.gin) -> gout_d.
template <int NC, int ST>
__global__ void convert_g(StepArgs A, const double* __restrict__ gin_d, double* __restrict__ gout_d,
                          bool to_storage) {
    using Real = typename StoreTraits<ST>::Real;
    const int nx = A.nx, ny = A.ny;
    const size_t nxy = (size_t)nx * ny;
    for (size_t node = blockIdx.x * (size_t)blockDim.x + threadIdx.x; node < nxy;
         node += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(node % nx), y = (int)(node / nx);
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            if (to_storage) {
                // storage at r holds g_a(r + e_a)
                const size_t src = (size_t)wrap(y + ey(a), ny) * nx + wrap(x + ex(a), nx);
#pragma unroll
                for (int i = 0; i < NC; ++i)
                    store_g<ST>(A, i, a, node, nxy, (Real)gin_d[(size_t)(i * 9 + a) * nxy + src]);
            } else {
                const size_t src = (size_t)wrap(y - ey(a), ny) * nx + wrap(x - ex(a), nx);
#pragma unroll
                for (int i = 0; i < NC; ++i)
                    gout_d[(size_t)(i * 9 + a) * nxy + node] = (double)load_g<ST>(A, i, a, src, nxy);
            }
        }
    }
}

// Deterministic reductions over a lattice: one thread per node on the same 32 x 8 tiling
// as the step (so the block count, and with it the summation order, depends only on
// the lattice shape).  Each block writes NC + 2 double sums: sum rho_i, sum (rho - rho_prev)^2,
// sum rho^2; then rho_prev <- rho.  reduce_final adds the block rows in a fixed order.
// A fused step asked for the diagnostics of the state it reads writes the same partial
// sums, bit for bit (same node sums, same shuffle tree, same strips).  The sums are exact
// to about 44 bits within a warp (float-float for float storage) and double from the
// strips up; rho_prev holds values of the storage arithmetic type.
constexpr int kRedTY = 8;

template <int NC, int ST>
__global__ void __launch_bounds__(kTX* kRedTY) reduce_partial(StepArgs A,
                                                               typename StoreTraits<ST>::Real* __restrict__ rho_prev,
                                                               int have_prev, double* __restrict__ partial) {
    using Real = typename StoreTraits<ST>::Real;
    const int nx = A.nx, ny = A.ny, nxy = nx * ny;
    const int x = blockIdx.x * kTX + threadIdx.x, y = blockIdx.y * kRedTY + threadIdx.y;
    Sum2<Real> acc[NC + 2];
#pragma unroll
    for (int k = 0; k < NC + 2; ++k) acc[k] = s2_of(Real(0));
    if (x < nx && y < ny) {
        const bool inner = x >= 1 && x + 1 < nx && y >= 1 && y + 1 < ny;
        Real pv[NC];
#pragma unroll
        for (int i = 0; i < NC; ++i) pv[i] = rho_prev[(size_t)i * nxy + (size_t)y * nx + x];
        Real r[NC];
        pull_rho<NC, ST>(A, x, y, inner, nx, ny, nxy, r);
        diag_node<NC, Real>(r, pv, have_prev, acc);
#pragma unroll
        for (int i = 0; i < NC; ++i) rho_prev[(size_t)i * nxy + (size_t)y * nx + x] = r[i];
    }
    __shared__ Sum2<Real> red[kRedTY][NC + 2];
    diag_warp<NC, Real>(acc, red[threadIdx.y]);
    __syncthreads();
    const int tid = threadIdx.y * kTX + threadIdx.x;
    if (tid < NC + 2)
        partial[(size_t)(blockIdx.y * gridDim.x + blockIdx.x) * (NC + 2) + tid] = diag_strip<NC, Real>(red, 0, tid, 0);
}

// Phase measure of a lattice: per component the sum over the nodes of ln rho_i, on the tiling
// of reduce_partial (NC double sums per 32 x 8 strip, compensated within a warp as there);
// sum_columns adds the strips in a fixed order.  Reads the state only.
template <int NC, int ST>
__global__ void __launch_bounds__(kTX* kRedTY) lnrho_partial(StepArgs A, double* __restrict__ partial) {
    using Real = typename StoreTraits<ST>::Real;
    const int nx = A.nx, ny = A.ny, nxy = nx * ny;
    const int x = blockIdx.x * kTX + threadIdx.x, y = blockIdx.y * kRedTY + threadIdx.y;
    Sum2<Real> acc[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) acc[k] = s2_of(Real(0));
    if (x < nx && y < ny) {
        const bool inner = x >= 1 && x + 1 < nx && y >= 1 && y + 1 < ny;
        Real r[NC];
        pull_rho<NC, ST>(A, x, y, inner, nx, ny, nxy, r);
        lnrho_node<NC, Real>(r, acc);
    }
    __shared__ Sum2<Real> red[kRedTY][NC];
    sums_warp<NC, Real>(acc, red[threadIdx.y]);
    __syncthreads();
    const int tid = threadIdx.y * kTX + threadIdx.x;
    if (tid < NC)
        partial[(size_t)(blockIdx.y * gridDim.x + blockIdx.x) * NC + tid] = sums_strip<NC, Real>(red, 0, tid, 0);
}

constexpr int kFinalThreads = 256;

// Column k of a table of nrows rows of K doubles, summed in double in a fixed order (strided
// over the threads, then a fixed tree); the result is valid in thread 0.
template <int K>
__device__ __forceinline__ double column_sum(const double* __restrict__ partial, int nrows, int k) {
    double v = 0.0;
    for (int b = threadIdx.x; b < nrows; b += kFinalThreads) v += partial[(size_t)b * K + k];
    __shared__ double red[kFinalThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kFinalThreads / 32; ++w) t += red[w];
    return t;
}

// latch (may be null): the handle's error latch, copied after the sums (at out + kMaxC + 2) so
// that one device-to-host copy brings a request's results and the error state together.
template <int NC>
__global__ void __launch_bounds__(kFinalThreads) reduce_final(const double* __restrict__ partial, int nblocks,
                                                               double* __restrict__ out,
                                                               const ErrorLatch* __restrict__ latch) {
    // block k sums quantity k over all strips
    const int k = blockIdx.x;
    if (latch != nullptr && k == 0 && threadIdx.x == 0) {
        const volatile int* src = reinterpret_cast<const volatile int*>(latch);
        int* dst = reinterpret_cast<int*>(out + kMaxC + 2);
#pragma unroll
        for (int q = 0; q < (int)(sizeof(ErrorLatch) / sizeof(int)); ++q) dst[q] = src[q];
    }
    const double t = column_sum<NC + 2>(partial, nblocks, k);
    if (threadIdx.x == 0) out[k] = t;
}

// out[k] = column k of a table of nrows rows of K doubles (one block per column).
template <int K>
__global__ void __launch_bounds__(kFinalThreads) sum_columns(const double* __restrict__ partial, int nrows,
                                                              double* __restrict__ out) {
    const double t = column_sum<K>(partial, nrows, blockIdx.x);
    if (threadIdx.x == 0) out[blockIdx.x] = t;
}

inline int reduce_blocks(int nx, int ny) { return ((nx + kTX - 1) / kTX) * ((ny + kRedTY - 1) / kRedTY); }

}  // namespace fmlbm
