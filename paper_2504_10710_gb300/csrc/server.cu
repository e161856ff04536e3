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
#include <list>
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

// FNV-1a over 64-bit words (then the tail bytes): the mesh key of a
// coordinate array, computed once per registered mesh.
unsigned long long fnv1a(const void* data, size_t n) {
    const unsigned char* p = static_cast<const unsigned char*>(data);
    unsigned long long h = 1469598103934665603ULL;
    size_t i = 0;
    for (; i + 8 <= n; i += 8) {
        unsigned long long w;
        std::memcpy(&w, p + i, 8);
        h ^= w;
        h *= 1099511628211ULL;
    }
    for (; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ULL;
    }
    return h;
}

// A mesh known to the server: its description with its own copy of the
// coordinates, key and memory estimate.  Requests point at it.
struct MeshRec {
    glls_mesh_desc desc{};
    std::vector<double> coords;
    MeshKey key;
    size_t estimate = 0;
    long long N = 0;
};

struct Request {
    unsigned long long id = 0;
    glls_mesh_desc desc{};
    std::vector<double> f, g;
    std::shared_ptr<const MeshRec> mesh;
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

// One instance of a resident mesh: the problem that set it up, or a clone
// sharing its mesh data with its own right-hand side and Krylov state.
struct Instance {
    glls_problem* prob = nullptr;
    bool busy = false;
};

// A resident mesh.  List nodes never move, so a worker may keep pointers to
// its mesh and instance while it holds the instance busy: eviction only
// removes meshes whose instances are all idle.
struct Cached {
    MeshKey key;
    std::list<Instance> inst;      // the set-up problem first, then clones
    size_t shared_bytes = 0;       // mesh data, held until the last instance goes
    size_t instance_bytes = 0;     // what each instance owns alone
    int cloning = 0;               // clones being created (their bytes are reserved)
    Clock::time_point last_used;
    bool idle() const {
        if (cloning) return false;
        for (const auto& i : inst)
            if (i.busy) return false;
        return true;
    }
    size_t bytes() const { return shared_bytes + inst.size() * instance_bytes; }
};

// What admit() hands a worker, decided under the server lock.
struct Admission {
    Request* r = nullptr;
    Cached* mesh = nullptr;        // resident mesh (run or clone), or null (create)
    glls_problem* prob = nullptr;  // idle instance taken, or null
    size_t reserve = 0;            // bytes reserved for a new mesh or clone
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
    std::list<Cached> cache;
    size_t resident = 0;     // bytes of cached meshes plus reservations being created
    unsigned long long next_id = 1, submitted = 0, completed = 0, failed = 0, running = 0, clones = 0;
    bool stop = false;
    std::vector<std::thread> workers;
    std::vector<MeshKey> creating;   // meshes whose set-up is in progress
    std::unordered_map<unsigned long long, std::shared_ptr<const MeshRec>> meshes;   // registered
    unsigned long long next_mesh = 1;

    bool pending_key(const MeshKey& k) const {
        for (const auto& c : creating)
            if (c == k) return true;
        return false;
    }

    Cached* find(const MeshKey& k) {
        for (auto& c : cache)
            if (c.key == k) return &c;
        return nullptr;
    }

    void finish_failed(Request* r, glls_status st) {
        r->status = st;
        r->state = 2;
        r->finished = Clock::now();
        ++failed;
        cv_done.notify_all();
    }

    // Evicts idle meshes other than `keep`, least recently used first, until
    // `need` more bytes fit the budget.  Returns whether they fit.
    bool make_room(size_t need, const Cached* keep) {
        while (resident + need > budget) {
            auto victim = cache.end();
            for (auto it = cache.begin(); it != cache.end(); ++it)
                if (&*it != keep && it->idle() && (victim == cache.end() || it->last_used < victim->last_used))
                    victim = it;
            if (victim == cache.end()) return false;
            for (auto& i : victim->inst) glls_problem_destroy(i.prob);
            resident -= victim->bytes();
            cache.erase(victim);
        }
        return true;
    }

    // Under the lock: the first queued request that can run now, in arrival
    // order.  A resident mesh with an idle instance runs on it; a resident
    // mesh whose instances are all busy gets a clone when its bytes fit (else
    // the request waits for an instance while later requests go ahead); a new
    // mesh reserves its estimate, evicting idle meshes; the oldest new-mesh
    // request that does not fit waits for memory and holds back the rest.
    bool admit(Admission* a) {
        for (auto it = queue.begin(); it != queue.end();) {
            Request* r = *it;
            Cached* c = find(r->key);
            if (c) {
                for (auto& i : c->inst)
                    if (!i.busy) {
                        i.busy = true;
                        *a = Admission{r, c, i.prob, 0};
                        queue.erase(it);
                        return true;
                    }
                if (make_room(c->instance_bytes, c)) {
                    resident += c->instance_bytes;
                    ++c->cloning;
                    *a = Admission{r, c, nullptr, c->instance_bytes};
                    queue.erase(it);
                    return true;
                }
                ++it;
                continue;
            }
            if (pending_key(r->key)) {
                ++it;
                continue;
            }
            if (r->estimate > budget) {       // can never fit: fail it here
                finish_failed(r, GLLS_ERR_BUDGET);
                it = queue.erase(it);
                continue;
            }
            if (!make_room(r->estimate, nullptr)) return false;
            resident += r->estimate;
            creating.push_back(r->key);
            *a = Admission{r, nullptr, nullptr, r->estimate};
            queue.erase(it);
            return true;
        }
        return false;
    }

    void worker() {
        cudaSetDevice(device);
        cudaStream_t stream = nullptr;
        cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
        for (;;) {
            Admission a;
            {
                std::unique_lock<std::mutex> lock(m);
                cv_work.wait(lock, [&] { return stop || admit(&a); });
                if (!a.r) break;
                a.r->state = 1;
                a.r->started = Clock::now();
                ++running;
            }
            Request* r = a.r;
            Cached* mesh = a.mesh;
            glls_problem* prob = a.prob;
            glls_status st = GLLS_OK;
            double setup_ms = 0.0;
            if (!prob && mesh) {
                // all instances of the resident mesh are busy: a clone shares its mesh data
                glls_problem* base = mesh->inst.front().prob;
                auto t0 = Clock::now();
                st = glls_problem_clone(base, &prob);
                setup_ms = std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
                std::lock_guard<std::mutex> lock(m);
                --mesh->cloning;
                resident -= a.reserve;
                if (st == GLLS_OK) {
                    glls_info inf;
                    glls_problem_info(prob, &inf);
                    Instance in;
                    in.prob = prob;
                    in.busy = true;
                    mesh->inst.push_back(in);
                    resident += mesh->instance_bytes;
                    ++clones;
                }
            } else if (!prob) {
                auto t0 = Clock::now();
                st = glls_problem_create(&r->desc, &prob);
                setup_ms = std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
                std::lock_guard<std::mutex> lock(m);
                resident -= a.reserve;
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
                    c.instance_bytes = inf.instance_bytes;
                    c.shared_bytes = inf.device_bytes - inf.instance_bytes;
                    Instance in;
                    in.prob = prob;
                    in.busy = true;
                    c.inst.push_back(in);
                    c.last_used = Clock::now();
                    cache.push_back(std::move(c));
                    mesh = &cache.back();
                    resident += mesh->bytes();
                }
            }
            // a new resident mesh or instance can admit waiting requests now
            if (!a.prob) cv_work.notify_all();
            glls_stats stats{};
            if (st == GLLS_OK) st = glls_set_rhs(prob, r->f.data(), 0, stream);
            if (st == GLLS_OK && !r->g.empty()) st = glls_set_dirichlet(prob, r->g.data(), 0, stream);
            if (st == GLLS_OK) st = glls_solve(prob, &r->opts, r->u, 0, stream, &stats);
            {
                std::lock_guard<std::mutex> lock(m);
                if (mesh) {
                    for (auto& i : mesh->inst)
                        if (i.prob == prob) i.busy = false;
                    mesh->last_used = Clock::now();
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
    for (auto& c : S->cache)
        for (auto& i : c.inst) glls_problem_destroy(i.prob);
    delete S;
}

static std::shared_ptr<MeshRec> make_mesh(glls_server* S, const glls_mesh_desc* mesh, glls_status* st) {
    auto m = std::make_shared<MeshRec>();
    *st = glls_estimate_bytes(mesh, &m->estimate);
    if (*st != GLLS_OK) return nullptr;
    long long N = 1;
    for (int a = 0; a < mesh->dim; ++a) N *= (long long)mesh->nelem[a] * mesh->order + 1;
    m->N = N;
    m->coords.assign(mesh->coords, mesh->coords + (size_t)mesh->dim * N);
    m->desc = *mesh;
    m->desc.coords = m->coords.data();
    m->desc.device = S->device;
    m->key.dim = mesh->dim;
    m->key.order = mesh->order;
    m->key.smoother = mesh->smoother;
    m->key.restriction = mesh->restriction;
    m->key.coarse_solver = mesh->coarse_solver;
    m->key.coarse_cr_levels = mesh->coarse_cr_levels;
    for (int a = 0; a < 3; ++a) m->key.nelem[a] = a < mesh->dim ? mesh->nelem[a] : 1;
    m->key.ncoords = m->coords.size();
    m->key.hash = fnv1a(m->coords.data(), sizeof(double) * m->coords.size());
    return m;
}

static glls_status enqueue(glls_server* S, std::shared_ptr<const MeshRec> m, const double* f, const double* g,
                           const glls_solve_opts* opts, double* u, unsigned long long* ticket) {
    auto r = std::make_unique<Request>();
    r->mesh = m;
    r->N = m->N;
    r->f.assign(f, f + m->N);
    if (g) r->g.assign(g, g + m->N);
    r->desc = m->desc;
    r->opts = *opts;
    r->u = u;
    r->estimate = m->estimate;
    r->key = m->key;
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

glls_status glls_submit(glls_server* S, const glls_mesh_desc* mesh, const double* f, const double* g,
                        const glls_solve_opts* opts, double* u, unsigned long long* ticket) {
    if (!S || !mesh || !f || !opts || !u || !ticket || !mesh->coords) return GLLS_ERR_INVALID;
    glls_status st = GLLS_OK;
    std::shared_ptr<MeshRec> m;
    try {
        m = make_mesh(S, mesh, &st);
    } catch (const std::bad_alloc&) {
        return GLLS_ERR_OOM;
    }
    if (!m) return st;
    return enqueue(S, m, f, g, opts, u, ticket);
}

glls_status glls_server_register(glls_server* S, const glls_mesh_desc* mesh, unsigned long long* mesh_id) {
    if (!S || !mesh || !mesh_id || !mesh->coords) return GLLS_ERR_INVALID;
    glls_status st = GLLS_OK;
    std::shared_ptr<MeshRec> m;
    try {
        m = make_mesh(S, mesh, &st);
    } catch (const std::bad_alloc&) {
        return GLLS_ERR_OOM;
    }
    if (!m) return st;
    std::lock_guard<std::mutex> lock(S->m);
    *mesh_id = S->next_mesh++;
    S->meshes.emplace(*mesh_id, std::move(m));
    return GLLS_OK;
}

glls_status glls_submit_mesh(glls_server* S, unsigned long long mesh_id, const double* f, const double* g,
                             const glls_solve_opts* opts, double* u, unsigned long long* ticket) {
    if (!S || !f || !opts || !u || !ticket) return GLLS_ERR_INVALID;
    std::shared_ptr<const MeshRec> m;
    {
        std::lock_guard<std::mutex> lock(S->m);
        auto it = S->meshes.find(mesh_id);
        if (it == S->meshes.end()) return GLLS_ERR_INVALID;
        m = it->second;
    }
    try {
        return enqueue(S, m, f, g, opts, u, ticket);
    } catch (const std::bad_alloc&) {
        return GLLS_ERR_OOM;
    }
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
    out->clones = S->clones;
    int inst = 0;
    for (const auto& c : S->cache) inst += (int)c.inst.size();
    out->cached_instances = inst;
    return GLLS_OK;
}

glls_status glls_cancel(glls_server* S, unsigned long long ticket) {
    if (!S) return GLLS_ERR_INVALID;
    {
        std::lock_guard<std::mutex> lock(S->m);
        auto it = S->requests.find(ticket);
        if (it == S->requests.end()) return GLLS_ERR_INVALID;
        Request* r = it->second.get();
        if (r->state != 0) return GLLS_NOT_READY;
        for (auto q = S->queue.begin(); q != S->queue.end(); ++q)
            if (*q == r) {
                S->queue.erase(q);
                break;
            }
        S->requests.erase(it);
    }
    S->cv_work.notify_all();
    return GLLS_OK;
}

}  // extern "C"
