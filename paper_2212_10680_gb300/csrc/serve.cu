// Serving (C ABI part of include/fmlbm.h): a request queue in front of a batch.
//
// A worker thread owns the batch and its stream.  Between chunks of steps it admits
// queued requests in arrival order while a slot is free and the requests' device
// bytes fit the budget (head-of-line: a request that does not fit waits for memory to
// free up, later ones wait behind it), runs one graph-captured chunk for every
// admitted lattice, checks residuals and phase measures, and retires each lattice at its own
// criterion (the configured measure below tol, a latched error, or its step limit), copying its final
// densities out and freeing its memory.  Each lattice's arithmetic is unaffected by
// what else runs (the batch guarantees bit-identical per-lattice results), so a
// request's result is the same alone and in any mix.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "fmlbm.h"

namespace {

double now_s(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

struct Pending {
    uint64_t id = 0, tag = 0;
    fmlbm_mixture mix{};
    fmlbm_lattice lat{};
    std::vector<double> rho;
    double* rho_out = nullptr;
    size_t bytes = 0;
    double t_submit = 0, t_admit = 0;
    int32_t slot = -1;
};

}  // namespace

struct fmlbm_server {
    fmlbm_server_config cfg{};
    int device = 0;
    cudaStream_t stream = nullptr;
    fmlbm_batch* batch = nullptr;
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Pending> queue;
    std::map<int32_t, Pending> running;  // by slot (worker only)
    int32_t running_count = 0;           // mirrored under mu
    std::vector<fmlbm_result> done;
    size_t bytes_admitted = 0;
    uint64_t next_id = 1;
    bool stop = false;
    double busy = 0;
    fmlbm_status worker_error = FMLBM_OK;
    std::string last_error;
    std::thread worker;
};

namespace {

void finish(fmlbm_server* s, Pending& p, int32_t status, int64_t steps, double residual, const double* liquid,
            const double* vapour) {
    fmlbm_result r;
    std::memset(&r, 0, sizeof r);
    r.id = p.id;
    r.tag = p.tag;
    r.status = status;
    r.n_components = p.mix.n_components;
    for (int i = 0; i < p.mix.n_components && liquid; ++i) {
        r.rho_liquid[i] = liquid[i];
        r.rho_vapour[i] = vapour[i];
    }
    r.steps = steps;
    r.residual = residual;
    r.t_submit = p.t_submit;
    r.t_admit = p.t_admit;
    r.t_done = now_s(s->t0);
    std::lock_guard<std::mutex> lock(s->mu);
    s->done.push_back(r);
    s->bytes_admitted -= p.bytes;
    s->running_count -= 1;
}

void worker_main(fmlbm_server* s) {
    cudaSetDevice(s->device);
    while (true) {
        // admission
        std::vector<Pending> admit;
        {
            std::unique_lock<std::mutex> lock(s->mu);
            if (s->running.empty() && s->queue.empty())
                s->cv.wait_for(lock, std::chrono::milliseconds(20), [&] { return s->stop || !s->queue.empty(); });
            if (s->stop) break;
            while (!s->queue.empty() && (int)(s->running.size() + admit.size()) < s->cfg.max_slots &&
                   s->bytes_admitted + s->queue.front().bytes <= s->cfg.hbm_budget_bytes) {
                s->bytes_admitted += s->queue.front().bytes;
                s->running_count += 1;
                admit.push_back(std::move(s->queue.front()));
                s->queue.pop_front();
            }
        }
        for (auto& p : admit) {
            int32_t slot = -1;
            fmlbm_status st = fmlbm_batch_add(s->batch, &p.mix, &p.lat, p.rho.data(), &slot);
            p.t_admit = now_s(s->t0);
            p.rho.clear();
            p.rho.shrink_to_fit();
            if (st != FMLBM_OK) {
                finish(s, p, st, 0, NAN, nullptr, nullptr);
                continue;
            }
            p.slot = slot;
            s->running.emplace(slot, std::move(p));
        }
        if (s->running.empty()) continue;
        // one chunk for every admitted lattice, then the per-lattice retirement check
        const double tb = now_s(s->t0);
        fmlbm_status st = fmlbm_batch_run_chunk(s->batch, s->cfg.chunk_steps);
        {
            std::lock_guard<std::mutex> lock(s->mu);
            s->busy += now_s(s->t0) - tb;
        }
        if (st != FMLBM_OK) {
            std::lock_guard<std::mutex> lock(s->mu);
            s->worker_error = st;
            s->last_error = fmlbm_batch_last_error(s->batch);
            s->stop = true;
            break;
        }
        std::vector<int32_t> retired;
        for (auto& kv : s->running) {
            int64_t steps = 0;
            double res = 0;
            int32_t status = 0, active = 0;
            fmlbm_batch_slot_info(s->batch, kv.first, &steps, &res, &status, &active);
            if (s->cfg.criterion == FMLBM_CRITERION_PHASE) fmlbm_batch_slot_phase_change(s->batch, kv.first, &res);
            bool retire = false;
            if (status != FMLBM_OK) retire = true;
            else if (res < s->cfg.tol) retire = true;
            else if (steps >= s->cfg.max_steps) {
                status = FMLBM_E_NOT_CONVERGED;
                retire = true;
            }
            if (!retire) continue;
            Pending& p = kv.second;
            double liquid[FMLBM_MAX_COMPONENTS] = {}, vapour[FMLBM_MAX_COMPONENTS] = {};
            const bool phases = status != FMLBM_E_NONPHYSICAL &&
                                fmlbm_batch_phases(s->batch, kv.first, liquid, vapour) == FMLBM_OK;
            if (p.rho_out && status != FMLBM_E_NONPHYSICAL)
                fmlbm_batch_moments(s->batch, kv.first, p.rho_out, nullptr, nullptr);
            fmlbm_batch_remove(s->batch, kv.first);
            finish(s, p, status, steps, res, phases ? liquid : nullptr, phases ? vapour : nullptr);
            retired.push_back(kv.first);
        }
        for (int32_t k : retired) s->running.erase(k);
    }
}

}  // namespace

extern "C" {

fmlbm_status fmlbm_server_create(const fmlbm_server_config* cfg, fmlbm_server** out) {
    if (!cfg || !out || cfg->max_slots < 1 || cfg->chunk_steps < 1 || cfg->max_steps < 1 || cfg->queue_capacity < 1 ||
        cfg->hbm_budget_bytes == 0 ||
        (cfg->criterion != FMLBM_CRITERION_RESIDUAL && cfg->criterion != FMLBM_CRITERION_PHASE))
        return FMLBM_E_INVALID_ARG;
    *out = nullptr;
    fmlbm_server* s = new (std::nothrow) fmlbm_server();
    if (!s) return FMLBM_E_OOM;
    s->cfg = *cfg;
    s->t0 = std::chrono::steady_clock::now();
    if (cudaGetDevice(&s->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete s;
        return FMLBM_E_CUDA;
    }
    fmlbm_status st = fmlbm_batch_create(cfg->n_components, cfg->precision, cfg->max_slots, s->stream, &s->batch);
    if (st != FMLBM_OK) {
        cudaStreamDestroy(s->stream);
        delete s;
        return st;
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return FMLBM_OK;
}

void fmlbm_server_destroy(fmlbm_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->device);
    fmlbm_batch_destroy(s->batch);
    cudaStreamDestroy(s->stream);
    delete s;
}

fmlbm_status fmlbm_server_submit(fmlbm_server* s, const fmlbm_request* req, uint64_t* id) {
    if (!s || !req || !req->rho) return FMLBM_E_INVALID_ARG;
    if (req->mixture.n_components != s->cfg.n_components || req->lattice.precision != s->cfg.precision)
        return FMLBM_E_INVALID_ARG;
    size_t bytes = 0;
    if (fmlbm_lattice_bytes(req->mixture.n_components, &req->lattice, &bytes) != FMLBM_OK) return FMLBM_E_INVALID_ARG;
    if (bytes > s->cfg.hbm_budget_bytes) return FMLBM_E_INVALID_ARG;  // could never be admitted
    Pending p;
    p.tag = req->tag;
    p.mix = req->mixture;
    p.lat = req->lattice;
    p.rho_out = req->rho_out;
    p.bytes = bytes;
    const size_t n = (size_t)req->mixture.n_components * req->lattice.nx * req->lattice.ny;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->stop) return s->worker_error != FMLBM_OK ? s->worker_error : FMLBM_E_INVALID_ARG;
        if ((int)s->queue.size() >= s->cfg.queue_capacity) return FMLBM_E_BUSY;
    }
    p.rho.assign(req->rho, req->rho + n);
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if ((int)s->queue.size() >= s->cfg.queue_capacity) return FMLBM_E_BUSY;
        p.id = s->next_id++;
        p.t_submit = now_s(s->t0);
        if (id) *id = p.id;
        s->queue.push_back(std::move(p));
    }
    s->cv.notify_one();
    return FMLBM_OK;
}

fmlbm_status fmlbm_server_poll(fmlbm_server* s, fmlbm_result* out, int32_t capacity, int32_t* n) {
    if (!s || !n || (capacity > 0 && !out)) return FMLBM_E_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    const int32_t k = (int32_t)std::min<size_t>(s->done.size(), (size_t)std::max(capacity, 0));
    for (int32_t q = 0; q < k; ++q) out[q] = s->done[q];
    s->done.erase(s->done.begin(), s->done.begin() + k);
    *n = k;
    return s->worker_error;
}

fmlbm_status fmlbm_server_stats(fmlbm_server* s, int32_t* queued, int32_t* running, size_t* bytes_admitted,
                                double* busy_seconds, double* now_seconds) {
    if (!s) return FMLBM_E_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    if (queued) *queued = (int32_t)s->queue.size();
    if (running) *running = s->running_count;
    if (bytes_admitted) *bytes_admitted = s->bytes_admitted;
    if (busy_seconds) *busy_seconds = s->busy;
    if (now_seconds) *now_seconds = now_s(s->t0);
    return s->worker_error;
}

}  // extern "C"
