// Serving runtime on top of the C ABI (include/glls.h): a request queue,
// worker slots with one CUDA stream each, a cache of resident problems keyed
// by the mesh, and admission by an HBM budget.  Requests are admitted in
// arrival order when a slot is free and the memory fits; admitted requests
// run concurrently on the device (continuous batching of independent solves).
#include "../../include/glls.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <functional>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

namespace {

using Clock = std::chrono::steady_clock;

struct MeshKey {
    int dim = 0, order = 0, smoother = 0, restriction = 0, coarse_solver = 0, coarse_cr_levels = 0;
    int nelem[3] = {1, 1, 1};
    size_t ncoords = 0;
    unsigned long long hash = 0;
    bool operator==(const MeshKey& o) const {
        return dim == o.dim && order == o.order && smoother == o.smoother && restriction == o.restriction &&
               coarse_solver == o.coarse_solver && coarse_cr_levels == o.coarse_cr_levels &&
               nelem[0] == o.nelem[0] && nelem[1] == o.nelem[1] && nelem[2] == o.nelem[2] &&
               ncoords == o.ncoords && hash == o.hash;
    }
};

unsigned long long fnv1a(const void* data, size_t n) {
    const unsigned char* p = static_cast<const unsigned char*>(data);
    unsigned long long h = 1469598103934665603ULL;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ULL;
    }
    return h;
}

struct Request {
    unsigned long long id = 0;
    glls_mesh_desc desc{};
    std::vector<double> coords, f, g;
    glls_solve_opts opts{};
    double* u = nullptr;
    MeshKey key;
    size_t estimate = 0;
    long long N = 0;
    int state = 0;                  // 0 queued, 1 running, 2 done
    glls_status status = GLLS_OK;
    glls_stats stats{};
    Clock::time_point submitted, started, finished;
};

struct Cached {
    MeshKey key;
    glls_problem* prob = nullptr;
    size_t bytes = 0;
    bool busy = false;
    Clock::time_point last_used;
};

}  // namespace

struct glls_server {
    int device = 0;
    size_t budget = 0;
    int nslots = 1;
    std::mutex m;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> queue;
    std::unordered_map<unsigned long long, std::unique_ptr<Request>> requests;
    std::vector<Cached> cache;
    size_t resident = 0;     // bytes of cached problems plus reservations being created
    unsigned long long next_id = 1, submitted = 0, completed = 0, failed = 0, running = 0;
    bool stop = false;
    std::vector<std::thread> workers;
    std::vector<MeshKey> creating;   // meshes whose set-up is in progress

    bool pending_key(const MeshKey& k) const {
        for (const auto& c : creating)
            if (c == k) return true;
        return false;
    }

    // Under the lock: choose the first queued request that can run now.
    // Returns it with `slot` set to a cached problem index, or -1 with
    // `reserve` bytes reserved for a new problem.  A request whose mesh is
    // resident but busy waits for that instance (no duplicate set-up) while
    // later requests for other meshes may proceed.
    Request* admit(int* slot, size_t* reserve) {
        for (auto it = queue.begin(); it != queue.end(); ++it) {
            Request* r = *it;
            bool resident_busy = false;
            for (size_t i = 0; i < cache.size(); ++i)
                if (cache[i].key == r->key) {
                    if (cache[i].busy) {
                        resident_busy = true;
                        continue;
                    }
                    cache[i].busy = true;
                    *slot = (int)i;
                    *reserve = 0;
                    queue.erase(it);
                    return r;
                }
            if (resident_busy || pending_key(r->key)) continue;
            if (r->estimate > budget) {       // can never fit: fail it here
                r->status = GLLS_ERR_BUDGET;
                r->state = 2;
                r->finished = Clock::now();
                ++failed;
                queue.erase(it);
                cv_done.notify_all();
                return admit(slot, reserve);
            }
            // evict idle cached problems, least recently used first, until it fits
            while (resident + r->estimate > budget) {
                int victim = -1;
                for (size_t i = 0; i < cache.size(); ++i)
                    if (!cache[i].busy && (victim < 0 || cache[i].last_used < cache[victim].last_used))
                        victim = (int)i;
                if (victim < 0) break;
                glls_problem_destroy(cache[victim].prob);
                resident -= cache[victim].bytes;
                cache.erase(cache.begin() + victim);
            }
            if (resident + r->estimate <= budget) {
                resident += r->estimate;
                *slot = -1;
                *reserve = r->estimate;
                creating.push_back(r->key);
                queue.erase(it);
                return r;
            }
            // the oldest request waits for memory: keep arrival order
            return nullptr;
        }
        return nullptr;
    }

    void worker() {
        cudaSetDevice(device);
        cudaStream_t stream = nullptr;
        cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
        for (;;) {
            Request* r = nullptr;
            int slot = -1;
            size_t reserve = 0;
            {
                std::unique_lock<std::mutex> lock(m);
                cv_work.wait(lock, [&] { return stop || (r = admit(&slot, &reserve)) != nullptr; });
                if (!r) break;
                r->state = 1;
                r->started = Clock::now();
                ++running;
            }
            glls_problem* prob = nullptr;
            glls_status st = GLLS_OK;
            double setup_ms = 0.0;
            if (slot >= 0) {
                std::lock_guard<std::mutex> lock(m);
                prob = cache[slot].prob;
            } else {
                auto t0 = Clock::now();
                st = glls_problem_create(&r->desc, &prob);
                setup_ms = std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
                std::lock_guard<std::mutex> lock(m);
                resident -= reserve;
                for (size_t i = 0; i < creating.size(); ++i)
                    if (creating[i] == r->key) {
                        creating.erase(creating.begin() + i);
                        break;
                    }
                if (st == GLLS_OK) {
                    glls_info inf;
                    glls_problem_info(prob, &inf);
                    Cached c;
                    c.key = r->key;
                    c.prob = prob;
                    c.bytes = inf.device_bytes;
                    c.busy = true;
                    cache.push_back(c);
                    resident += c.bytes;
                    slot = (int)cache.size() - 1;
                }
            }
            glls_stats stats{};
            if (st == GLLS_OK) st = glls_set_rhs(prob, r->f.data(), 0, stream);
            if (st == GLLS_OK && !r->g.empty()) st = glls_set_dirichlet(prob, r->g.data(), 0, stream);
            if (st == GLLS_OK) st = glls_solve(prob, &r->opts, r->u, 0, stream, &stats);
            {
                std::lock_guard<std::mutex> lock(m);
                for (auto& c : cache)
                    if (c.prob == prob) {
                        c.busy = false;
                        c.last_used = Clock::now();
                    }
                r->finished = Clock::now();
                stats.setup_ms = setup_ms;
                stats.solve_ms = std::chrono::duration<double, std::milli>(r->finished - r->submitted).count();
                stats.status = st;
                r->stats = stats;
                r->status = st;
                r->state = 2;
                --running;
                if (st == GLLS_OK) ++completed; else ++failed;
            }
            cv_done.notify_all();
            cv_work.notify_all();
        }
        cudaStreamDestroy(stream);
    }
};

extern "C" {

glls_status glls_server_create(int device, size_t hbm_budget_bytes, int slots, glls_server** out) {
    if (!out || slots < 1 || slots > 64 || hbm_budget_bytes == 0) return GLLS_ERR_INVALID;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return GLLS_ERR_CUDA;
    auto* S = new glls_server();
    S->device = device;
    S->budget = hbm_budget_bytes;
    S->nslots = slots;
    for (int i = 0; i < slots; ++i) S->workers.emplace_back([S] { S->worker(); });
    *out = S;
    return GLLS_OK;
}

void glls_server_destroy(glls_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lock(S->m);
        S->stop = true;
    }
    S->cv_work.notify_all();
    for (auto& t : S->workers) t.join();
    cudaSetDevice(S->device);
    for (auto& c : S->cache) glls_problem_destroy(c.prob);
    delete S;
}

glls_status glls_submit(glls_server* S, const glls_mesh_desc* mesh, const double* f, const double* g,
                        const glls_solve_opts* opts, double* u, unsigned long long* ticket) {
    if (!S || !mesh || !f || !opts || !u || !ticket || !mesh->coords) return GLLS_ERR_INVALID;
    auto r = std::make_unique<Request>();
    size_t est = 0;
    glls_status st = glls_estimate_bytes(mesh, &est);
    if (st != GLLS_OK) return st;
    long long N = 1;
    for (int a = 0; a < mesh->dim; ++a) N *= (long long)mesh->nelem[a] * mesh->order + 1;
    r->N = N;
    r->coords.assign(mesh->coords, mesh->coords + (size_t)mesh->dim * N);
    r->f.assign(f, f + N);
    if (g) r->g.assign(g, g + N);
    r->desc = *mesh;
    r->desc.coords = r->coords.data();
    r->desc.device = S->device;
    r->opts = *opts;
    r->u = u;
    r->estimate = est;
    r->key.dim = mesh->dim;
    r->key.order = mesh->order;
    r->key.smoother = mesh->smoother;
    r->key.restriction = mesh->restriction;
    r->key.coarse_solver = mesh->coarse_solver;
    r->key.coarse_cr_levels = mesh->coarse_cr_levels;
    for (int a = 0; a < 3; ++a) r->key.nelem[a] = a < mesh->dim ? mesh->nelem[a] : 1;
    r->key.ncoords = r->coords.size();
    r->key.hash = fnv1a(r->coords.data(), sizeof(double) * r->coords.size());
    r->submitted = Clock::now();
    {
        std::lock_guard<std::mutex> lock(S->m);
        r->id = S->next_id++;
        *ticket = r->id;
        S->queue.push_back(r.get());
        S->requests.emplace(r->id, std::move(r));
        ++S->submitted;
    }
    S->cv_work.notify_all();
    return GLLS_OK;
}

glls_status glls_poll(glls_server* S, unsigned long long ticket, int wait, glls_stats* stats) {
    if (!S) return GLLS_ERR_INVALID;
    std::unique_lock<std::mutex> lock(S->m);
    auto it = S->requests.find(ticket);
    if (it == S->requests.end()) return GLLS_ERR_INVALID;
    Request* r = it->second.get();
    if (r->state != 2) {
        if (!wait) return GLLS_NOT_READY;
        S->cv_done.wait(lock, [&] { return r->state == 2; });
    }
    if (stats) *stats = r->stats;
    const glls_status st = r->status;
    S->requests.erase(it);
    return st;
}

glls_status glls_server_info_get(glls_server* S, glls_server_info* out) {
    if (!S || !out) return GLLS_ERR_INVALID;
    std::lock_guard<std::mutex> lock(S->m);
    out->submitted = S->submitted;
    out->completed = S->completed;
    out->failed = S->failed;
    out->queued = S->queue.size();
    out->running = S->running;
    out->resident_bytes = S->resident;
    out->budget_bytes = S->budget;
    out->cached_problems = (int)S->cache.size();
    return GLLS_OK;
}

}  // extern "C"
