// Domain decomposition of one periodic lattice into y-slabs (C ABI part of include/fmlbm.h).
//
// The streaming of Eq. eqLBEMCa (Section III.B, step 9) is periodic; a lattice split into
// slabs along y needs, before each step, the rows of its neighbours that its update reads.
// The fused step reads, for a node, the distributions up to three rows away (the pulls of
// its 2-node halo of rho~), so each slab keeps three ghost rows above and below its own
// rows, in its own buffers: a slab of R rows is a lattice of R + 6 rows, stepped by the
// ordinary fused step.  Its own rows then compute exactly what the whole lattice computes
// (same inputs, same arithmetic); the ghost rows are overwritten after every step by the
// neighbours' boundary rows -- plain cudaMemcpy2DAsync copies of every distribution plane
// (one copy per plane group and neighbour), the halo exchange a multi-GPU split does with
// peer copies.  The ghost rows' own update (from pulls that wrap around the slab) is
// discarded, so the domain check of each slab covers its own rows only.  Here every slab
// lives on the current device.
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "fmlbm.h"
#include "fmlbm_internal.h"

namespace {

constexpr int kGhost = 3;  // rows a slab's update reads beyond its own: pull of the 2-node halo

struct Slab {
    fmlbm_handle* h = nullptr;
    void* g[2] = {nullptr, nullptr};
    float* g0[2] = {nullptr, nullptr};
    void* F[2] = {nullptr, nullptr};
};

}  // namespace

struct fmlbm_decomp {
    int nc = 0, nslabs = 0;
    fmlbm_lattice global{}, local{};
    int rows = 0;            // own rows per slab
    cudaStream_t stream = nullptr;
    std::vector<Slab> slab;
    int64_t steps = 0;       // steps since init: buffer (steps & 1) holds the state
    size_t esize = 0;        // bytes per element of the g planes
    int gplanes = 0;         // planes of g (9N, or 8N for the deviation forms)
    int g0planes = 0;        // float a = 0 planes (N for the deviation forms, else 0)
    std::string last_error;
};

namespace {

fmlbm_status dfail(fmlbm_decomp* d, fmlbm_status s, const std::string& m) {
    if (d) d->last_error = m;
    return s;
}

bool dev16(int precision) {
    return precision == FMLBM_FP16DEV || precision == FMLBM_BF16DEV || precision == FMLBM_FP16DEV_LNF64 ||
           precision == FMLBM_BF16DEV_LNF64;
}

void release(fmlbm_decomp* d) {
    for (Slab& s : d->slab) {
        if (s.h) fmlbm_destroy(s.h);
        for (int k = 0; k < 2; ++k) {
            if (s.g[k]) cudaFree(s.g[k]);
            if (s.g0[k]) cudaFree(s.g0[k]);
            if (s.F[k]) cudaFree(s.F[k]);
        }
    }
}

// Rows [src_row, src_row + 3) of every plane of slab `from` into rows [dst_row, dst_row + 3)
// of slab `to`, buffer b.  Planes are nx * (rows + 6) elements apart in both.
cudaError_t copy_rows(fmlbm_decomp* d, int from, int src_row, int to, int dst_row, int b) {
    const size_t nx = (size_t)d->local.nx, ny = (size_t)d->local.ny;
    const size_t pitch = nx * ny * d->esize, width = kGhost * nx * d->esize;
    const size_t so = (size_t)src_row * nx * d->esize, dO = (size_t)dst_row * nx * d->esize;
    cudaError_t e = cudaMemcpy2DAsync(static_cast<char*>(d->slab[to].g[b]) + dO, pitch,
                                      static_cast<const char*>(d->slab[from].g[b]) + so, pitch, width, d->gplanes,
                                      cudaMemcpyDefault, d->stream);
    if (e != cudaSuccess || !d->g0planes) return e;
    const size_t p4 = nx * ny * 4, w4 = kGhost * nx * 4;
    return cudaMemcpy2DAsync(reinterpret_cast<char*>(d->slab[to].g0[b]) + (size_t)dst_row * nx * 4, p4,
                             reinterpret_cast<const char*>(d->slab[from].g0[b]) + (size_t)src_row * nx * 4, p4, w4,
                             d->g0planes, cudaMemcpyDefault, d->stream);
}

// Ghost rows of every slab from its neighbours' own boundary rows, buffer b: rows 0..2 of
// slab s take own rows R..R+2 (its last three) of slab s - 1; rows R+3..R+5 take own rows
// 3..5 (its first three) of slab s + 1 (periodic in the slab index).
cudaError_t exchange(fmlbm_decomp* d, int b) {
    const int n = d->nslabs, R = d->rows;
    for (int s = 0; s < n; ++s) {
        cudaError_t e = copy_rows(d, (s - 1 + n) % n, R, s, 0, b);
        if (e == cudaSuccess) e = copy_rows(d, (s + 1) % n, kGhost, s, R + kGhost, b);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

extern "C" {

fmlbm_status fmlbm_decomp_slab_rows(int32_t ny, int32_t nslabs, int32_t slab, int32_t* y0, int32_t* rows) {
    if (!y0 || !rows || nslabs < 1 || ny < 1 || slab < 0 || slab >= nslabs || ny % nslabs != 0 ||
        ny / nslabs < kGhost)
        return FMLBM_E_INVALID_ARG;
    *rows = ny / nslabs;
    *y0 = slab * *rows;
    return FMLBM_OK;
}

fmlbm_status fmlbm_decomp_create(const fmlbm_mixture* mixture, const fmlbm_lattice* lattice, int32_t nslabs,
                                 void* cuda_stream, fmlbm_decomp** out) {
    if (!mixture || !lattice || !out || nslabs < 1) return FMLBM_E_INVALID_ARG;
    *out = nullptr;
    int32_t y0 = 0, rows = 0;
    if (fmlbm_decomp_slab_rows(lattice->ny, nslabs, 0, &y0, &rows) != FMLBM_OK) return FMLBM_E_INVALID_ARG;
    std::string why;
    if (!fmlbm_internal_lattice_ok(*lattice, mixture->n_components, &why)) return FMLBM_E_INVALID_ARG;
    fmlbm_decomp* d = new (std::nothrow) fmlbm_decomp();
    if (!d) return FMLBM_E_OOM;
    d->nc = mixture->n_components;
    d->nslabs = nslabs;
    d->global = *lattice;
    d->local = *lattice;
    d->local.ny = rows + 2 * kGhost;
    d->rows = rows;
    d->stream = static_cast<cudaStream_t>(cuda_stream);
    d->gplanes = dev16(lattice->precision) ? 8 * d->nc : 9 * d->nc;
    d->g0planes = dev16(lattice->precision) ? d->nc : 0;
    d->esize = dev16(lattice->precision) ? 2 : (lattice->precision == FMLBM_FP64 ? 8 : 4);
    size_t gb = 0, g0b = 0, fb = 0;
    if (fmlbm_buffer_sizes(d->nc, &d->local, &gb, &g0b, &fb) != FMLBM_OK) {
        delete d;
        return FMLBM_E_INVALID_ARG;
    }
    d->slab.resize(nslabs);
    for (Slab& s : d->slab) {
        bool ok = true;
        for (int k = 0; k < 2 && ok; ++k) {
            ok = cudaMalloc(&s.g[k], gb) == cudaSuccess && cudaMalloc(&s.F[k], fb) == cudaSuccess;
            if (ok && g0b) ok = cudaMalloc((void**)&s.g0[k], g0b) == cudaSuccess;
        }
        fmlbm_status st = ok ? fmlbm_create_with_buffers(mixture, &d->local, cuda_stream, s.g, g0b ? s.g0 : nullptr,
                                                         s.F, &s.h)
                             : FMLBM_E_OOM;
        if (st != FMLBM_OK) {
            cudaGetLastError();
            release(d);
            delete d;
            return st;
        }
        fmlbm_internal_set_check_rows(s.h, kGhost, kGhost + rows);
    }
    *out = d;
    return FMLBM_OK;
}

fmlbm_status fmlbm_decomp_init(fmlbm_decomp* d, const double* rho_host) {
    if (!d || !rho_host) return dfail(d, FMLBM_E_INVALID_ARG, "null argument");
    const size_t nx = (size_t)d->global.nx, ny = (size_t)d->global.ny, nyl = (size_t)d->local.ny;
    std::vector<double> local((size_t)d->nc * nyl * nx);
    for (int s = 0; s < d->nslabs; ++s) {
        // the slab's own rows and its ghost rows (periodic in y)
        for (int i = 0; i < d->nc; ++i)
            for (size_t r = 0; r < nyl; ++r) {
                const long long gy = ((long long)s * d->rows + (long long)r - kGhost + (long long)ny) % (long long)ny;
                std::memcpy(&local[((size_t)i * nyl + r) * nx], rho_host + ((size_t)i * ny + (size_t)gy) * nx,
                            nx * sizeof(double));
            }
        fmlbm_status st = fmlbm_init(d->slab[s].h, local.data());
        if (st != FMLBM_OK) return dfail(d, st, std::string("slab init: ") + fmlbm_last_error(d->slab[s].h));
    }
    d->steps = 0;
    return FMLBM_OK;
}

fmlbm_status fmlbm_decomp_step(fmlbm_decomp* d, int64_t nsteps) {
    if (!d || nsteps < 0) return dfail(d, FMLBM_E_INVALID_ARG, "bad argument");
    for (int64_t k = 0; k < nsteps; ++k) {
        for (int s = 0; s < d->nslabs; ++s) {
            fmlbm_status st = fmlbm_step(d->slab[s].h, 1);
            if (st != FMLBM_OK) return dfail(d, st, fmlbm_last_error(d->slab[s].h));
        }
        ++d->steps;
        // the state is now in buffer (steps & 1) of every slab: refresh its ghost rows
        cudaError_t e = exchange(d, (int)(d->steps & 1));
        if (e != cudaSuccess) return dfail(d, FMLBM_E_CUDA, std::string("halo exchange: ") + cudaGetErrorString(e));
    }
    return FMLBM_OK;
}

fmlbm_status fmlbm_decomp_get_distributions(fmlbm_decomp* d, double* g_host, double* force_host) {
    if (!d) return FMLBM_E_INVALID_ARG;
    const size_t nx = (size_t)d->global.nx, ny = (size_t)d->global.ny, nyl = (size_t)d->local.ny;
    std::vector<double> g(g_host ? (size_t)d->nc * 9 * nyl * nx : 0), F(force_host ? 2 * nyl * nx : 0);
    for (int s = 0; s < d->nslabs; ++s) {
        fmlbm_status st = fmlbm_get_distributions(d->slab[s].h, g_host ? g.data() : nullptr,
                                                  force_host ? F.data() : nullptr);
        if (st != FMLBM_OK) return dfail(d, st, fmlbm_last_error(d->slab[s].h));
        for (size_t r = 0; r < (size_t)d->rows; ++r) {
            const size_t gy = (size_t)s * d->rows + r, ly = r + kGhost;
            for (size_t p = 0; g_host && p < (size_t)d->nc * 9; ++p)
                std::memcpy(g_host + (p * ny + gy) * nx, &g[(p * nyl + ly) * nx], nx * sizeof(double));
            for (size_t p = 0; force_host && p < 2; ++p)
                std::memcpy(force_host + (p * ny + gy) * nx, &F[(p * nyl + ly) * nx], nx * sizeof(double));
        }
    }
    return FMLBM_OK;
}

const char* fmlbm_decomp_last_error(const fmlbm_decomp* d) { return d ? d->last_error.c_str() : ""; }

void fmlbm_decomp_destroy(fmlbm_decomp* d) {
    if (!d) return;
    if (d->stream) cudaStreamSynchronize(d->stream);
    else cudaDeviceSynchronize();
    release(d);
    delete d;
}

}  // extern "C"
