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
    int dim = 0, order = 0, smoother = 0, restriction = 0, coarse_solver = 0, coarse_cr_levels = 0, summation = 0;
    int nelem[3] = {1, 1, 1};
    size_t ncoords = 0;
    unsigned long long hash = 0;
    bool operator==(const MeshKey& o) const {
        return dim == o.dim && order == o.order && smoother == o.smoother && restriction == o.restriction &&
               coarse_solver == o.coarse_solver && coarse_cr_levels == o.coarse_cr_levels &&
               summation == o.summation && nelem[0] == o.nelem[0] && nelem[1] == o.nelem[1] && nelem[2] == o.nelem[2] &&
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
    std::vector<double> f, g;          // owned copies (glls_submit)
    const double* fp = nullptr;        // the data read by the solve: the copies, or the
    const double* gp = nullptr;        // caller's buffers (glls_submit_mesh)
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
// sharing its mesh data with its own right-hand sides and Krylov state.
struct Instance {
    glls_problem* prob = nullptr;
    int nrhs = 1;                  // right-hand sides it solves together
    size_t bytes = 0;              // device memory it owns alone
    bool busy = false;
};

// A resident mesh.  List nodes never move, so a worker may keep pointers to
// its mesh and instance while it holds the instance busy: eviction only
// removes meshes whose instances are all idle.
struct Cached {
    MeshKey key;
    std::list<Instance> inst;      // the set-up problem first, then clones
    size_t shared_bytes = 0;       // mesh data, held until the last instance goes
    size_t instance_bytes = 0;     // what a one-right-hand-side instance owns alone
    int cloning = 0;               // clones being created (their bytes are reserved)
    Clock::time_point last_used;
    bool idle() const {
        if (cloning) return false;
        for (const auto& i : inst)
            if (i.busy) return false;
        return true;
    }
    size_t bytes() const {
        size_t b = shared_bytes;
        for (const auto& i : inst) b += i.bytes;
        return b;
    }
};

// What admit() hands a worker, decided under the server lock: requests of
// one mesh solved together (one, or a group sharing Dirichlet data and
// options when grouping is on).
struct Admission {
    std::vector<Request*> rs;
    Cached* mesh = nullptr;        // resident mesh (run or clone), or null (create)
    glls_problem* prob = nullptr;  // idle instance taken, or null
    int nrhs = 1;                  // right-hand sides of the instance
    size_t reserve = 0;            // bytes reserved for a new mesh or clone
};

bool same_opts(const glls_solve_opts& a, const glls_solve_opts& b) {
    return a.tol == b.tol && a.max_iter == b.max_iter && a.gamma == b.gamma && a.m == b.m && a.alpha == b.alpha &&
           a.precision == b.precision && a.krylov == b.krylov && a.use_graph == b.use_graph &&
           a.check_every == b.check_every;
}

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
    int max_group = 1;               // requests solved together (1: no grouping)
    unsigned long long grouped = 0;  // requests served by multi-right-hand-side solves

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
    // With grouping (max_group > 1), queued requests of a resident mesh that
    // share its Dirichlet data and options are taken together, up to the
    // largest power of two <= max_group available, and solved as one
    // multi-right-hand-side solve on an instance of that size.
    bool admit(Admission* a) {
        for (auto it = queue.begin(); it != queue.end();) {
            Request* r = *it;
            Cached* c = find(r->key);
            if (c) {
                std::vector<std::deque<Request*>::iterator> grp{it};
                if (max_group > 1 && r->opts.use_graph == 2 && r->opts.krylov != GLLS_KRYLOV_GMRES)
                    for (auto jt = std::next(it); jt != queue.end() && (int)grp.size() < max_group; ++jt)
                        if ((*jt)->key == r->key && (*jt)->gp == r->gp && same_opts((*jt)->opts, r->opts))
                            grp.push_back(jt);
                int g = 1;
                while (2 * g <= (int)grp.size()) g *= 2;
                for (; g >= 1; g /= 2) {
                    Instance* idle = nullptr;
                    for (auto& i : c->inst)
                        if (!i.busy && i.nrhs == g) {
                            idle = &i;
                            break;
                        }
                    size_t need = 0;
                    if (!idle) {
                        need = c->instance_bytes * (size_t)g;
                        if (!make_room(need, c)) continue;
                        resident += need;
                        ++c->cloning;
                    } else {
                        idle->busy = true;
                    }
                    *a = Admission{{}, c, idle ? idle->prob : nullptr, g, need};
                    for (int k = 0; k < g; ++k) a->rs.push_back(*grp[k]);
                    // one pass over the queue (erasing inside a deque invalidates its iterators)
                    queue.erase(std::remove_if(queue.begin(), queue.end(),
                                               [&](Request* q) {
                                                   return std::find(a->rs.begin(), a->rs.end(), q) != a->rs.end();
                                               }),
                                queue.end());
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
            *a = Admission{{r}, nullptr, nullptr, 1, r->estimate};
            queue.erase(it);
            return true;
        }
        return false;
    }

    void worker() {
        cudaSetDevice(device);
        cudaStream_t stream = nullptr;
        cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
        std::vector<double> F, U;                 // staging of a group's right-hand sides and solutions
        std::vector<glls_stats> st_all;
        for (;;) {
            Admission a;
            {
                std::unique_lock<std::mutex> lock(m);
                cv_work.wait(lock, [&] { return stop || admit(&a); });
                if (a.rs.empty()) break;
                for (Request* q : a.rs) {
                    q->state = 1;
                    q->started = Clock::now();
                }
                running += a.rs.size();
            }
            Request* r = a.rs.front();
            const int g = (int)a.rs.size();
            Cached* mesh = a.mesh;
            glls_problem* prob = a.prob;
            glls_status st = GLLS_OK;
            double setup_ms = 0.0;
            int setup_kind = prob ? 0 : mesh ? 2 : 1;
            if (!prob && mesh) {
                // no idle instance of this size: a clone shares the mesh data
                glls_problem* base = mesh->inst.front().prob;
                auto t0 = Clock::now();
                st = glls_problem_clone_nrhs(base, a.nrhs, &prob);
                setup_ms = std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
                std::lock_guard<std::mutex> lock(m);
                --mesh->cloning;
                resident -= a.reserve;
                if (st == GLLS_OK) {
                    glls_info inf;
                    glls_problem_info(prob, &inf);
                    Instance in;
                    in.prob = prob;
                    in.nrhs = a.nrhs;
                    in.bytes = inf.instance_bytes;
                    in.busy = true;
                    mesh->inst.push_back(in);
                    resident += in.bytes;
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
                    in.bytes = inf.instance_bytes;
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
            st_all.assign(g, glls_stats{});
            if (g == 1) {
                if (st == GLLS_OK) st = glls_set_rhs(prob, r->fp, 0, stream);
                if (st == GLLS_OK && r->gp) st = glls_set_dirichlet(prob, r->gp, 0, stream);
                if (st == GLLS_OK) st = glls_solve(prob, &r->opts, r->u, 0, stream, st_all.data());
                st_all[0].status = st;
            } else {
                const size_t N = (size_t)r->N;
                try {
                    F.resize(N * g);
                    U.resize(N * g);
                } catch (const std::bad_alloc&) {
                    st = GLLS_ERR_OOM;
                }
                if (st == GLLS_OK) {
                    for (int k = 0; k < g; ++k) std::memcpy(&F[N * k], a.rs[k]->fp, sizeof(double) * N);
                    st = glls_set_rhs(prob, F.data(), 0, stream);
                }
                if (st == GLLS_OK && r->gp) st = glls_set_dirichlet(prob, r->gp, 0, stream);
                if (st == GLLS_OK) {
                    glls_solve(prob, &r->opts, U.data(), 0, stream, st_all.data());   // per-RHS status in st_all
                    for (int k = 0; k < g; ++k) std::memcpy(a.rs[k]->u, &U[N * k], sizeof(double) * N);
                } else {
                    for (auto& x : st_all) x.status = st;
                }
            }
            {
                std::lock_guard<std::mutex> lock(m);
                if (mesh) {
                    for (auto& i : mesh->inst)
                        if (i.prob == prob) i.busy = false;
                    mesh->last_used = Clock::now();
                }
                const auto done = Clock::now();
                for (int k = 0; k < g; ++k) {
                    Request* q = a.rs[k];
                    glls_stats& s = st_all[k];
                    q->finished = done;
                    s.setup_ms = k == 0 ? setup_ms : 0.0;
                    s.setup_kind = k == 0 ? setup_kind : 0;
                    s.group = g;
                    s.queue_ms = std::chrono::duration<double, std::milli>(q->started - q->submitted).count();
                    s.solve_ms = std::chrono::duration<double, std::milli>(q->finished - q->submitted).count();
                    q->stats = s;
                    q->status = (glls_status)s.status;
                    q->state = 2;
                    if (s.status == GLLS_OK) ++completed; else ++failed;
                }
                running -= g;
                grouped += g > 1 ? g : 0;
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
    m->key.summation = mesh->summation;
    for (int a = 0; a < 3; ++a) m->key.nelem[a] = a < mesh->dim ? mesh->nelem[a] : 1;
    m->key.ncoords = m->coords.size();
    m->key.hash = fnv1a(m->coords.data(), sizeof(double) * m->coords.size());
    return m;
}

// copy = true: f and g are copied now; else the request reads the caller's
// buffers when it runs.
static glls_status enqueue(glls_server* S, std::shared_ptr<const MeshRec> m, const double* f, const double* g,
                           const glls_solve_opts* opts, double* u, unsigned long long* ticket, bool copy) {
    auto r = std::make_unique<Request>();
    r->mesh = m;
    r->N = m->N;
    if (copy) {
        r->f.assign(f, f + m->N);
        if (g) r->g.assign(g, g + m->N);
        r->fp = r->f.data();
        r->gp = g ? r->g.data() : nullptr;
    } else {
        r->fp = f;
        r->gp = g;
    }
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
    return enqueue(S, m, f, g, opts, u, ticket, true);
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
        return enqueue(S, m, f, g, opts, u, ticket, false);
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

glls_status glls_server_set_max_group(glls_server* S, int max_group) {
    if (!S || max_group < 1 || max_group > 64) return GLLS_ERR_INVALID;
    std::lock_guard<std::mutex> lock(S->m);
    S->max_group = max_group;
    return GLLS_OK;
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
    out->grouped = S->grouped;
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
