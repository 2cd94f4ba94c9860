// Continuous-batching solve server (mrhs_server_* / mrhs_submit / mrhs_poll).
//
// Each resident hierarchy (config) owns a fixed block of `slots` RHS columns
// on the device and one worker thread with its own CUDA stream, so the
// solves of different configs overlap on the GPU.  A worker repeatedly
//   1. admits queued requests (FIFO) whose columns fit into free slots and
//      whose device staging (its sources, later its solution columns) fits
//      into free HBM above the server's reserve (cudaMemGetInfo at each
//      admission; the staging is allocated then and freed when the request
//      completes): their sources are copied into the slot columns, their x
//      set to zero;
//   2. runs the MG-preconditioned FP64 FGMRES on the whole slot block for at
//      most one restart cycle (outer_m iterations), stopping early once some
//      column has converged while requests are waiting;
//   3. retires every column whose true residual met its request's tolerance,
//      copying its solution out and freeing the slot.
// Because every RHS has its own Krylov space (independent per-column
// recurrences, batched kernels), a request's result does not depend on which
// other requests shared its batch beyond the fixed reduction order.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "mg.cuh"

namespace mrhs {
mrhs_status api_record(mrhs_status code, const std::string &msg);
}

using namespace mrhs;

namespace {

using Clock = std::chrono::steady_clock;

// column c of a [rows][n] field
__global__ void k_scatter_cols(double2 *__restrict__ dst, int dst_n, const double2 *__restrict__ src, int src_n,
                               const int *__restrict__ slot_of, int64_t rows) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * src_n) return;
    const int64_t row = i / src_n;
    const int c = (int)(i - row * src_n);
    dst[row * dst_n + slot_of[c]] = src[i];
}

__global__ void k_gather_cols(double2 *__restrict__ dst, int dst_n, const double2 *__restrict__ src, int src_n,
                              const int *__restrict__ slot_of, int64_t rows) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * dst_n) return;
    const int64_t row = i / dst_n;
    const int c = (int)(i - row * dst_n);
    dst[i] = src[row * src_n + slot_of[c]];
}

__global__ void k_zero_cols(double2 *__restrict__ f, int n, const int *__restrict__ slot_of, int k, int64_t rows) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * k) return;
    const int64_t row = i / k;
    const int c = (int)(i - row * k);
    f[row * n + slot_of[c]] = make_double2(0.0, 0.0);
}

struct Request {
    uint64_t id = 0;
    int config = 0;
    int nrhs = 0;
    double tol = 0;
    std::vector<double2> b;  // host copy of the sources [rows][nrhs]
    double *x_host = nullptr;
    DeviceBuffer dev;        // device staging [rows][nrhs] FP64, held from admission to completion
    mrhs_status state = MRHS_PENDING;
    Clock::time_point t_submit, t_admit, t_done;
    bool admitted = false;
    int cols_done = 0;
    int outer_iters = 0;
    double max_rel = 0;
    std::string error;
};

struct Slot {
    uint64_t req = 0;  // 0: free
    int col = 0;       // column of the request
    int cycles = 0;
};

struct Config {
    mrhs_mg *mg = nullptr;
    int slots = 0;
    int64_t rows = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    DeviceBuffer b, x;        // FP64 [rows][slots]
    DeviceBuffer slot_map;    // int [slots]
    std::vector<Slot> table;
    std::deque<uint64_t> queue;
    std::thread worker;
};

}  // namespace

struct mrhs_server {
    mrhs_server_params p{};
    std::mutex mu;
    std::condition_variable cv;       // wakes workers
    std::condition_variable done_cv;  // wakes drain / waiters
    std::map<uint64_t, Request> reqs;
    std::vector<std::unique_ptr<Config>> configs;
    std::atomic<bool> stop{false};
    uint64_t next_id = 1;
    int outstanding = 0;
    uint64_t mem_waits = 0;  // admissions deferred (or refused) for lack of free HBM
    int staged = 0;          // requests holding device staging
    static constexpr int kMaxCycles = 64;  // restart cycles a column may take before failing
};

namespace {

void finish_request(mrhs_server &srv, Request &r, mrhs_status st, const std::string &err) {
    r.state = st;
    r.error = err;
    r.t_done = Clock::now();
    if (r.dev.ptr) srv.staged--;
    r.dev.release();
    std::vector<double2>().swap(r.b);
    srv.outstanding--;
    srv.done_cv.notify_all();
    srv.cv.notify_all();
}

void worker_loop(mrhs_server *srv, Config *cfg) {
    cudaSetDevice(cfg->device);
    const int S = cfg->slots;
    const int64_t rows = cfg->rows;
    std::vector<double> tols(S, 0.5), rel(S, 0.0);
    std::vector<int> map(S);
    while (true) {
        // ---- admission
        std::vector<std::pair<uint64_t, std::vector<int>>> admitted;
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            auto busy = [&] {
                for (const Slot &sl : cfg->table)
                    if (sl.req) return true;
                return false;
            };
            srv->cv.wait(lk, [&] { return srv->stop.load() || !cfg->queue.empty() || busy(); });
            if (srv->stop.load()) return;
            while (!cfg->queue.empty()) {
                Request &r = srv->reqs[cfg->queue.front()];
                std::vector<int> free_slots;
                for (int s = 0; s < S && (int)free_slots.size() < r.nrhs; ++s)
                    if (!cfg->table[s].req) free_slots.push_back(s);
                if ((int)free_slots.size() < r.nrhs) break;  // FIFO: wait for room
                // memory admission: the request's device staging must fit into free HBM
                // above the reserve; otherwise it waits for running requests to free
                // theirs, and fails only if nothing else holds memory here
                const size_t need = sizeof(double2) * (size_t)rows * r.nrhs;
                size_t free_b = 0, total_b = 0;
                bool fits = cudaMemGetInfo(&free_b, &total_b) == cudaSuccess &&
                            (double)free_b >= (double)need + srv->p.hbm_reserve_gb * 1e9;
                if (fits) {
                    try {
                        r.dev.alloc(need);
                    } catch (const std::exception &) {
                        (void)cudaGetLastError();
                        fits = false;
                    }
                }
                if (!fits) {
                    srv->mem_waits++;
                    if (srv->staged > 0) break;  // memory held by running requests will come back
                    cfg->queue.pop_front();
                    finish_request(*srv, r, MRHS_ERR_OOM, "not enough free HBM to stage the request");
                    continue;
                }
                srv->staged++;
                for (int c = 0; c < r.nrhs; ++c) cfg->table[free_slots[c]] = Slot{r.id, c, 0};
                r.admitted = true;
                r.t_admit = Clock::now();
                admitted.emplace_back(r.id, free_slots);
                cfg->queue.pop_front();
            }
            if (admitted.empty() && !busy()) {
                // nothing runs on this config: its head request waits for slots or HBM
                // that requests of other configs hold; look again shortly
                srv->cv.wait_for(lk, std::chrono::milliseconds(2));
                continue;
            }
        }
        try {
            // ---- load the admitted sources into their slots
            for (auto &a : admitted) {
                const Request *rq;
                {
                    std::lock_guard<std::mutex> lk(srv->mu);
                    rq = &srv->reqs[a.first];
                }
                const int k = (int)a.second.size();
                MRHS_CUDA(cudaMemcpyAsync(cfg->slot_map.ptr, a.second.data(), sizeof(int) * k, cudaMemcpyHostToDevice,
                                          cfg->stream));
                MRHS_CUDA(cudaMemcpyAsync(rq->dev.ptr, rq->b.data(), sizeof(double2) * rows * k,
                                          cudaMemcpyHostToDevice, cfg->stream));
                k_scatter_cols<<<ceil_div(rows * k, 256), 256, 0, cfg->stream>>>(
                    cfg->b.as<double2>(), S, rq->dev.as<double2>(), k, cfg->slot_map.as<int>(), rows);
                k_zero_cols<<<ceil_div(rows * k, 256), 256, 0, cfg->stream>>>(cfg->x.as<double2>(), S,
                                                                              cfg->slot_map.as<int>(), k, rows);
                MRHS_LAUNCHED("server scatter");
                MRHS_CUDA(cudaStreamSynchronize(cfg->stream));
                std::lock_guard<std::mutex> lk(srv->mu);
                std::vector<double2>().swap(srv->reqs[a.first].b);  // sources now live on the device
            }
            // ---- one restart cycle on the whole slot block
            {
                std::lock_guard<std::mutex> lk(srv->mu);
                for (int s = 0; s < S; ++s)
                    tols[s] = cfg->table[s].req ? srv->reqs[cfg->table[s].req].tol : 0.5;
            }
            auto stop_early = [&](const double *relest, int n) {
                std::lock_guard<std::mutex> lk(srv->mu);
                if (cfg->queue.empty()) return false;
                for (int s = 0; s < n; ++s)
                    if (cfg->table[s].req && relest[s] <= 0.5 * tols[s]) return true;
                return false;
            };
            mrhs_solve_stats st{};
            mg_solve(*cfg->mg, cfg->b.as<double2>(), cfg->x.as<double2>(), S, tols.data(), rel.data(), &st,
                     cfg->stream, std::max(1, mg_outer_m(cfg->mg)), stop_early);
            // ---- retire converged columns
            std::vector<std::pair<uint64_t, std::vector<int>>> to_copy;  // (req, slots in column order)
            {
                std::lock_guard<std::mutex> lk(srv->mu);
                std::map<uint64_t, std::vector<int>> fin;
                for (int s = 0; s < S; ++s) {
                    Slot &sl = cfg->table[s];
                    if (!sl.req) continue;
                    Request &r = srv->reqs[sl.req];
                    if (sl.col == 0) r.outer_iters += st.outer_iters;
                    sl.cycles++;
                    if (rel[s] <= r.tol) {
                        r.max_rel = std::max(r.max_rel, rel[s]);
                        fin[sl.req].push_back(s);
                    } else if (sl.cycles >= mrhs_server::kMaxCycles) {
                        r.max_rel = std::max(r.max_rel, rel[s]);
                        fin[sl.req].push_back(s);
                        r.error = "column did not converge within the cycle cap";
                    }
                }
                for (auto &kv : fin) to_copy.emplace_back(kv.first, kv.second);
            }
            for (auto &tc : to_copy) {
                Request *rq;
                {
                    std::lock_guard<std::mutex> lk(srv->mu);
                    rq = &srv->reqs[tc.first];
                }
                // copy each finished column to the request's x (columns are interleaved on the host)
                const int k = (int)tc.second.size();
                MRHS_CUDA(cudaMemcpyAsync(cfg->slot_map.ptr, tc.second.data(), sizeof(int) * k, cudaMemcpyHostToDevice,
                                          cfg->stream));
                k_gather_cols<<<ceil_div(rows * k, 256), 256, 0, cfg->stream>>>(
                    rq->dev.as<double2>(), k, cfg->x.as<double2>(), S, cfg->slot_map.as<int>(), rows);
                MRHS_LAUNCHED("server gather");
                std::vector<double2> host((size_t)rows * k);
                MRHS_CUDA(cudaMemcpyAsync(host.data(), rq->dev.ptr, sizeof(double2) * rows * k,
                                          cudaMemcpyDeviceToHost, cfg->stream));
                MRHS_CUDA(cudaStreamSynchronize(cfg->stream));
                std::vector<int> cols(k);
                {
                    std::lock_guard<std::mutex> lk(srv->mu);
                    for (int c = 0; c < k; ++c) cols[c] = cfg->table[tc.second[c]].col;
                }
                double2 *xo = reinterpret_cast<double2 *>(rq->x_host);
                for (int64_t row = 0; row < rows; ++row)
                    for (int c = 0; c < k; ++c) xo[row * rq->nrhs + cols[c]] = host[(size_t)row * k + c];
                std::lock_guard<std::mutex> lk(srv->mu);
                for (int c = 0; c < k; ++c) cfg->table[tc.second[c]] = Slot{};
                k_zero_cols<<<ceil_div(rows * k, 256), 256, 0, cfg->stream>>>(cfg->b.as<double2>(), S,
                                                                              cfg->slot_map.as<int>(), k, rows);
                k_zero_cols<<<ceil_div(rows * k, 256), 256, 0, cfg->stream>>>(cfg->x.as<double2>(), S,
                                                                              cfg->slot_map.as<int>(), k, rows);
                MRHS_CUDA(cudaStreamSynchronize(cfg->stream));
                rq->cols_done += k;
                if (rq->cols_done == rq->nrhs)
                    finish_request(*srv, *rq, rq->error.empty() ? MRHS_OK : MRHS_ERR_NOT_CONVERGED, rq->error);
            }
        } catch (const std::exception &e) {
            // fail every request that holds a slot; keep serving the queue
            std::lock_guard<std::mutex> lk(srv->mu);
            for (Slot &sl : cfg->table) {
                if (!sl.req) continue;
                Request &r = srv->reqs[sl.req];
                if (r.state == MRHS_PENDING) finish_request(*srv, r, MRHS_ERR_CUDA, e.what());
                sl = Slot{};
            }
            cudaMemsetAsync(cfg->b.ptr, 0, cfg->b.bytes, cfg->stream);
            cudaMemsetAsync(cfg->x.ptr, 0, cfg->x.bytes, cfg->stream);
            cudaStreamSynchronize(cfg->stream);
        }
    }
}

#define S_TRY try {
#define S_CATCH                                                                     \
    }                                                                               \
    catch (const mrhs::Error &e) { return api_record(e.code, e.what()); }           \
    catch (const std::bad_alloc &) { return api_record(MRHS_ERR_OOM, "host allocation failed"); } \
    catch (const std::exception &e) { return api_record(MRHS_ERR_CUDA, e.what()); }

}  // namespace

extern "C" {

mrhs_status mrhs_server_create(const mrhs_server_params *params, mrhs_server **out) {
    S_TRY
    if (!params || !out) fail(MRHS_ERR_INVALID, "params and out must be non-null");
    if (params->max_queue < 1) fail(MRHS_ERR_INVALID, "max_queue must be >= 1");
    if (params->hbm_reserve_gb < 0) fail(MRHS_ERR_INVALID, "hbm_reserve_gb must be >= 0");
    auto srv = std::make_unique<mrhs_server>();
    srv->p = *params;
    *out = srv.release();
    api_record(MRHS_OK, "");
    return MRHS_OK;
    S_CATCH
}

mrhs_status mrhs_server_add_config(mrhs_server *srv, mrhs_mg *mg, int slots, int *config_id) {
    S_TRY
    if (!srv || !mg || !config_id) fail(MRHS_ERR_INVALID, "server, mg and config_id must be non-null");
    if (slots < 1 || slots > mg_max_rhs(mg)) fail(MRHS_ERR_INVALID, "slots must be in 1..max_rhs of the hierarchy");
    auto cfg = std::make_unique<Config>();
    cfg->mg = mg;
    cfg->slots = slots;
    cfg->rows = mg_fine_rows(mg);
    cfg->device = mg_device(mg);
    MRHS_CUDA(cudaSetDevice(cfg->device));
    const size_t field = sizeof(double2) * (size_t)cfg->rows * slots;
    size_t free_b = 0, total_b = 0;
    MRHS_CUDA(cudaMemGetInfo(&free_b, &total_b));
    const double need = 2.0 * field + srv->p.hbm_reserve_gb * 1e9;
    if ((double)free_b < need)
        fail(MRHS_ERR_OOM, "not enough free HBM to admit this configuration");
    cfg->b.alloc(field);
    cfg->x.alloc(field);
    cfg->slot_map.alloc(sizeof(int) * slots);
    MRHS_CUDA(cudaMemset(cfg->b.ptr, 0, field));
    MRHS_CUDA(cudaMemset(cfg->x.ptr, 0, field));
    MRHS_CUDA(cudaStreamCreateWithFlags(&cfg->stream, cudaStreamNonBlocking));
    cfg->table.assign(slots, Slot{});
    Config *raw = cfg.get();
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->configs.push_back(std::move(cfg));
        *config_id = (int)srv->configs.size() - 1;
    }
    raw->worker = std::thread(worker_loop, srv, raw);
    api_record(MRHS_OK, "");
    return MRHS_OK;
    S_CATCH
}

mrhs_status mrhs_submit(mrhs_server *srv, int config_id, const double *b_host, double *x_host, int nrhs, double tol,
                        uint64_t *req_id) {
    S_TRY
    if (!srv || !b_host || !x_host || !req_id) fail(MRHS_ERR_INVALID, "non-null server, b, x and req_id required");
    if (!(tol > 0 && tol < 1)) fail(MRHS_ERR_INVALID, "tol must be in (0, 1)");
    std::unique_lock<std::mutex> lk(srv->mu);
    if (config_id < 0 || config_id >= (int)srv->configs.size()) fail(MRHS_ERR_INVALID, "unknown config");
    Config *cfg = srv->configs[config_id].get();
    if (nrhs < 1 || nrhs > cfg->slots) fail(MRHS_ERR_INVALID, "nrhs must be in 1..slots of the config");
    if ((int)cfg->queue.size() >= srv->p.max_queue) fail(MRHS_ERR_BUSY, "request queue full");
    {
        // a request whose staging cannot fit even into the whole device above the reserve never will
        size_t free_b = 0, total_b = 0;
        MRHS_CUDA(cudaSetDevice(cfg->device));
        MRHS_CUDA(cudaMemGetInfo(&free_b, &total_b));
        const double need = (double)sizeof(double2) * (double)cfg->rows * nrhs;
        if (need + srv->p.hbm_reserve_gb * 1e9 > (double)total_b)
            fail(MRHS_ERR_OOM, "request staging exceeds the device memory above the reserve");
    }
    Request r;
    r.id = srv->next_id++;
    r.config = config_id;
    r.nrhs = nrhs;
    r.tol = tol;
    r.x_host = x_host;
    r.t_submit = Clock::now();
    lk.unlock();
    // copy sources column-block wise: host layout [rows][nrhs] is already what the stage expects
    std::vector<double2> b((size_t)cfg->rows * nrhs);
    std::memcpy(b.data(), b_host, sizeof(double2) * b.size());
    lk.lock();
    r.b = std::move(b);
    const uint64_t id = r.id;
    srv->reqs.emplace(id, std::move(r));
    cfg->queue.push_back(id);
    srv->outstanding++;
    *req_id = id;
    srv->cv.notify_all();
    api_record(MRHS_OK, "");
    return MRHS_OK;
    S_CATCH
}

mrhs_status mrhs_server_set_reserve(mrhs_server *srv, double hbm_reserve_gb) {
    S_TRY
    if (!srv) fail(MRHS_ERR_INVALID, "server must be non-null");
    if (!(hbm_reserve_gb >= 0)) fail(MRHS_ERR_INVALID, "hbm_reserve_gb must be >= 0");
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->p.hbm_reserve_gb = hbm_reserve_gb;
    }
    srv->cv.notify_all();
    api_record(MRHS_OK, "");
    return MRHS_OK;
    S_CATCH
}

mrhs_status mrhs_server_memory_waits(mrhs_server *srv, uint64_t *count) {
    S_TRY
    if (!srv || !count) fail(MRHS_ERR_INVALID, "server and count must be non-null");
    std::lock_guard<std::mutex> lk(srv->mu);
    *count = srv->mem_waits;
    api_record(MRHS_OK, "");
    return MRHS_OK;
    S_CATCH
}

mrhs_status mrhs_poll(mrhs_server *srv, uint64_t req_id, mrhs_request_stats *stats) {
    S_TRY
    if (!srv) fail(MRHS_ERR_INVALID, "server must be non-null");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(req_id);
    if (it == srv->reqs.end()) return api_record(MRHS_ERR_NOT_FOUND, "unknown request id");
    const Request &r = it->second;
    if (stats) {
        stats->state = r.state;
        const auto now = Clock::now();
        stats->latency_s = std::chrono::duration<double>((r.state == MRHS_PENDING ? now : r.t_done) - r.t_submit).count();
        stats->queue_s = r.admitted ? std::chrono::duration<double>(r.t_admit - r.t_submit).count() : stats->latency_s;
        stats->outer_iters = r.outer_iters;
        stats->max_rel_residual = r.max_rel;
    }
    if (r.state == MRHS_PENDING) {
        api_record(MRHS_OK, "");
        return MRHS_PENDING;
    }
    if (r.state != MRHS_OK) return api_record(r.state, r.error);
    api_record(MRHS_OK, "");
    return MRHS_OK;
    S_CATCH
}

mrhs_status mrhs_server_drain(mrhs_server *srv) {
    S_TRY
    if (!srv) fail(MRHS_ERR_INVALID, "server must be non-null");
    std::unique_lock<std::mutex> lk(srv->mu);
    srv->done_cv.wait(lk, [&] { return srv->outstanding == 0; });
    api_record(MRHS_OK, "");
    return MRHS_OK;
    S_CATCH
}

void mrhs_server_destroy(mrhs_server *srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv.notify_all();
    for (auto &c : srv->configs)
        if (c->worker.joinable()) c->worker.join();
    for (auto &c : srv->configs)
        if (c->stream) {
            cudaSetDevice(c->device);
            cudaStreamSynchronize(c->stream);
            cudaStreamDestroy(c->stream);
        }
    delete srv;
}

}  // extern "C"
