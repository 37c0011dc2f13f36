// wx_ensemble.cu -- batched ensembles of uneven grids stepped by one
// persistent launch per step (replayed from a captured CUDA graph), and the
// launch-configuration autotuner shared by single contexts and ensembles.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <new>
#include <sstream>

#include "wx_internal.cuh"

using namespace wx;

struct wx_ens {
    std::vector<wx_ctx *> mem;
    int dtype = 0;
    StepCfg cfg;
    bool cfg_forced = false;
    unsigned *d_status = nullptr;
    cudaStream_t capture_stream = nullptr;
    cudaStream_t last_stream = nullptr;
    struct Graph {
        int n_steps;
        unsigned parity, generation;
        StepCfg cfg;
        cudaGraphExec_t exec;
    };
    std::vector<Graph> graphs;
    long last_launches = 0;
    std::string err;
};

static thread_local std::string g_ens_create_error;

static int efail(wx_ens *e, int code, const std::string &m) {
    if (e)
        e->err = m;
    else
        g_ens_create_error = m;
    return code;
}

static unsigned parity_of(const wx_ens *e) {
    unsigned p = 0;
    for (size_t i = 0; i < e->mem.size(); ++i) p |= (unsigned)e->mem[i]->cur << i;
    return p;
}

static unsigned generation_of(const wx_ens *e) {
    unsigned g = 0;
    for (auto *c : e->mem) g = g * 2654435761u + c->generation;
    return g;
}

static void drop_graphs(wx_ens *e) {
    for (auto &g : e->graphs) cudaGraphExecDestroy(g.exec);
    e->graphs.clear();
}

static int nz_max_member(const wx_ens *e) {
    int k = 0;
    for (size_t i = 1; i < e->mem.size(); ++i)
        if (e->mem[i]->nz > e->mem[k]->nz) k = (int)i;
    return k;
}

// The configuration must fit the member with the deepest columns (its
// shared-memory plan is the largest); every member's TMA descriptors are
// re-encoded for the tile rows and planes per box.
static int ens_apply_cfg(wx_ens *e, const StepCfg &g) {
    if (!cfg_fits(e->mem[nz_max_member(e)], g, nullptr))
        return efail(e, WX_EUNSUPPORTED, "step configuration does not fit the deepest member");
    for (auto *c : e->mem) {
        const int rc = apply_cfg(c, g);
        if (rc != WX_OK) return efail(e, rc, c->err);
    }
    e->cfg = g;
    drop_graphs(e);
    return WX_OK;
}

extern "C" int wx_ens_create(int m, const int *nx, const int *ny, const int *nz, int dtype, wx_ens **out) {
    if (!out) return efail(nullptr, WX_EINVAL, "wx_ens_create: out is NULL");
    *out = nullptr;
    if (m < 1 || m > kMaxMembers) return efail(nullptr, WX_EINVAL, "wx_ens_create: 1..16 members");
    if (!nx || !ny || !nz) return efail(nullptr, WX_EINVAL, "wx_ens_create: NULL size array");
    if (dtype != WX_F32 && dtype != WX_F64) return efail(nullptr, WX_EUNSUPPORTED, "wx_ens_create: WX_F32 or WX_F64");
    wx_ens *e = new (std::nothrow) wx_ens();
    if (!e) return efail(nullptr, WX_ENOMEM, "wx_ens_create: host allocation failed");
    e->dtype = dtype;
    for (int i = 0; i < m; ++i) {
        wx_ctx *c = nullptr;
        const int rc = wx_create(nx[i], ny[i], nz[i], dtype, &c);
        if (rc != WX_OK) {
            g_ens_create_error = std::string("member ") + std::to_string(i) + ": " + wx_last_error(nullptr);
            wx_ens_destroy(e);
            return rc;
        }
        e->mem.push_back(c);
    }
    if (cudaMalloc(&e->d_status, sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(e->d_status, 0, sizeof(unsigned)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&e->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
        g_ens_create_error = "wx_ens_create: CUDA set-up failed";
        wx_ens_destroy(e);
        return WX_ECUDA;
    }
    const int rc = ens_apply_cfg(e, default_cfg(e->mem[nz_max_member(e)]));
    if (rc != WX_OK) {
        g_ens_create_error = e->err;
        wx_ens_destroy(e);
        return rc;
    }
    *out = e;
    return WX_OK;
}

extern "C" void wx_ens_destroy(wx_ens *e) {
    if (!e) return;
    drop_graphs(e);
    for (auto *c : e->mem) wx_destroy(c);
    if (e->d_status) cudaFree(e->d_status);
    if (e->capture_stream) cudaStreamDestroy(e->capture_stream);
    delete e;
}

extern "C" const char *wx_ens_last_error(const wx_ens *e) { return e ? e->err.c_str() : g_ens_create_error.c_str(); }

extern "C" wx_ctx *wx_ens_member(wx_ens *e, int i) {
    if (!e || i < 0 || i >= (int)e->mem.size()) return nullptr;
    return e->mem[i];
}

extern "C" int wx_ens_size(const wx_ens *e) { return e ? (int)e->mem.size() : 0; }

extern "C" long wx_ens_last_launches(const wx_ens *e) { return e ? e->last_launches : -1; }

// Checks before a batched step: every member set up, same options.
static int ens_ready(wx_ens *e) {
    const wx_ctx *c0 = e->mem[0];
    for (size_t i = 0; i < e->mem.size(); ++i) {
        wx_ctx *c = e->mem[i];
        if (!c->params_set || !c->fields_loaded)
            return efail(e, WX_ESTATE, "member " + std::to_string(i) + ": set params and load fields first");
        if (c->flags != c0->flags || (c->kmult != nullptr) != (c0->kmult != nullptr))
            return efail(e, WX_EINVAL, "members must share the option flags and kappa_mult use");
        if (c->flags & (WX_SURROGATE | WX_RK3))
            return efail(e, WX_EUNSUPPORTED, "WX_SURROGATE and WX_RK3 members step with wx_step, not in a batch");
        if (c->cfg.ty != e->cfg.ty || c->cfg.kb != e->cfg.kb) {
            const int rc = apply_cfg(c, e->cfg);
            if (rc != WX_OK) return efail(e, rc, c->err);
        }
        const int rc = check_cfl(c);
        if (rc != WX_OK) return efail(e, rc, "member " + std::to_string(i) + ": " + c->err);
    }
    return WX_OK;
}

static int ens_launch_steps(wx_ens *e, int n, cudaStream_t s, long *launches) {
    for (int k = 0; k < n; ++k) {
        const int rc = launch_batch(e->mem.data(), (int)e->mem.size(), e->cfg, e->d_status, s, launches, e->err);
        if (rc != WX_OK) return rc;
    }
    return WX_OK;
}

extern "C" int wx_ens_step(wx_ens *e, int n_steps, int use_graph, void *stream) {
    if (!e) return WX_EINVAL;
    if (n_steps < 0) return efail(e, WX_EINVAL, "wx_ens_step: n_steps < 0");
    int rc = ens_ready(e);
    if (rc != WX_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    e->last_stream = s;
    long launches = 0;
    if (!use_graph || n_steps == 0) {
        rc = ens_launch_steps(e, n_steps, s, &launches);
        e->last_launches = launches;
        return rc;
    }
    // one graph per (steps, buffer parities, member generations, config)
    const unsigned par = parity_of(e), gen = generation_of(e);
    wx_ens::Graph *hit = nullptr;
    for (auto &g : e->graphs)
        if (g.n_steps == n_steps && g.parity == par && g.generation == gen && g.cfg.ty == e->cfg.ty &&
            g.cfg.kb == e->cfg.kb && g.cfg.stages == e->cfg.stages && g.cfg.ctas_per_sm == e->cfg.ctas_per_sm &&
            g.cfg.prefetch == e->cfg.prefetch)
            hit = &g;
    std::vector<int> cur0(e->mem.size());
    for (size_t i = 0; i < e->mem.size(); ++i) cur0[i] = e->mem[i]->cur;
    if (!hit) {
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(e->capture_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return efail(e, WX_ECUDA, "wx_ens_step: stream capture failed to start");
        rc = ens_launch_steps(e, n_steps, e->capture_stream, &launches);
        const cudaError_t ce = cudaStreamEndCapture(e->capture_stream, &graph);
        for (size_t i = 0; i < e->mem.size(); ++i) e->mem[i]->cur = cur0[i];  // nothing ran yet
        if (rc != WX_OK || ce != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return rc != WX_OK ? rc : efail(e, WX_ECUDA, "wx_ens_step: stream capture failed");
        }
        cudaGraphExec_t exec = nullptr;
        const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) return efail(e, WX_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ie));
        e->graphs.push_back({n_steps, par, gen, e->cfg, exec});
        hit = &e->graphs.back();
        e->last_launches = launches;
    }
    const cudaError_t le = cudaGraphLaunch(hit->exec, s);
    if (le != cudaSuccess) return efail(e, WX_ECUDA, std::string("graph launch: ") + cudaGetErrorString(le));
    for (size_t i = 0; i < e->mem.size(); ++i) e->mem[i]->cur = cur0[i] ^ (n_steps & 1);
    return WX_OK;
}

extern "C" int wx_ens_sync(wx_ens *e) {
    if (!e) return WX_EINVAL;
    if (cudaStreamSynchronize(e->last_stream) != cudaSuccess) return efail(e, WX_ECUDA, "wx_ens_sync");
    unsigned st = 0;
    if (cudaMemcpy(&st, e->d_status, sizeof st, cudaMemcpyDeviceToHost) != cudaSuccess)
        return efail(e, WX_ECUDA, "wx_ens_sync: status");
    if (st) cudaMemset(e->d_status, 0, sizeof st);
    // members report non-finite values through their own status words
    for (size_t i = 0; i < e->mem.size(); ++i) {
        e->mem[i]->last_stream = e->last_stream;
        const int rc = wx_sync(e->mem[i]);
        if (rc != WX_OK) return efail(e, rc, "member " + std::to_string(i) + ": " + e->mem[i]->err);
    }
    if (st & ST_TIMEOUT) return efail(e, WX_ETIMEOUT, "a bounded device wait timed out");
    if (st & ST_BOUNDS) return efail(e, WX_ECUDA, "a kernel skipped an out-of-bounds access (bounds-checked build)");
    return WX_OK;
}

extern "C" int wx_ens_set_step_config(wx_ens *e, int ty, int kb, int stages, int ctas_per_sm, int prefetch) {
    if (!e) return WX_EINVAL;
    StepCfg g;
    g.ty = ty;
    g.kb = kb;
    g.stages = stages;
    g.ctas_per_sm = ctas_per_sm;
    g.prefetch = prefetch;
    if (!(ty == 1 || ty == 2 || ty == 4 || ty == 8 || ty == 12) || !(kb == 2 || kb == 4) || (ty == 1 && kb == 4) ||
        stages < 3 || stages > 16 || ctas_per_sm < 1 || prefetch < 0 || prefetch > 64)
        return efail(e, WX_EINVAL, "wx_ens_set_step_config: invalid configuration");
    const int rc = ens_apply_cfg(e, g);
    if (rc == WX_OK) e->cfg_forced = true;
    return rc;
}

extern "C" int wx_ens_get_step_config(const wx_ens *e, int *ty, int *kb, int *stages, int *ctas, int *prefetch) {
    if (!e) return WX_EINVAL;
    if (ty) *ty = e->cfg.ty;
    if (kb) *kb = e->cfg.kb;
    if (stages) *stages = e->cfg.stages;
    if (ctas) *ctas = e->cfg.ctas_per_sm;
    if (prefetch) *prefetch = e->cfg.prefetch;
    return WX_OK;
}

// ------------------------------------------------------------- autotuner
// Candidate launch shapes for a batch: tile rows x planes per box x ring
// slots, with the most CTAs per SM that fit and one fewer; each is timed
// with CUDA events over a few steps after a warm-up step, on copies of the
// members' states that are restored afterwards.  The winner is cached in a
// text file, one line per (GPU, dtype, options, member sizes).
static std::string tune_key(wx_ctx *const *mem, int n) {
    cudaDeviceProp p;
    cudaGetDeviceProperties(&p, mem[0]->device);
    std::ostringstream k;
    for (const char *q = p.name; *q; ++q) k << (*q == ' ' ? '_' : *q);
    k << "|dt" << mem[0]->dtype << "|f" << mem[0]->flags << "|km" << (mem[0]->kmult != nullptr);
    for (int i = 0; i < n; ++i) k << "|" << mem[i]->nx << "x" << mem[i]->ny << "x" << mem[i]->nz;
    return k.str();
}

static bool cache_lookup(const char *path, const std::string &key, StepCfg &g, double &ms) {
    if (!path || !*path) return false;
    std::ifstream f(path);
    std::string line;
    bool found = false;
    while (std::getline(f, line)) {
        std::istringstream is(line);
        std::string k;
        StepCfg c;
        double t;
        if (is >> k >> c.ty >> c.kb >> c.stages >> c.ctas_per_sm >> c.prefetch >> t && k == key) {
            g = c;
            ms = t;
            found = true;  // the last entry for a key wins
        }
    }
    return found;
}

static void cache_store(const char *path, const std::string &key, const StepCfg &g, double ms) {
    if (!path || !*path) return;
    std::ofstream f(path, std::ios::app);
    f << key << " " << g.ty << " " << g.kb << " " << g.stages << " " << g.ctas_per_sm << " " << g.prefetch << " " << ms
      << "\n";
}

// Tunes the batch `mem` (members already set up) and leaves the best
// configuration applied through `apply` (a single context or an ensemble).
template <typename Apply>
static int tune_batch(wx_ctx *const *mem, int n, unsigned *status, const char *cache, int force,
                      cudaStream_t s, Apply apply, StepCfg &best, double &best_ms, std::string &err) {
    const std::string key = tune_key(mem, n);
    if (!force && cache_lookup(cache, key, best, best_ms)) return apply(best);
    // snapshot the current states (the trials step the members)
    std::vector<void *> snap(n, nullptr);
    std::vector<int> cur0(n);
    std::vector<long long> cnt0(n);
    auto restore_and_free = [&](int rc) {
        for (int i = 0; i < n; ++i) {
            if (!snap[i]) continue;
            const size_t bytes = mem[i]->field_cells * mem[i]->cell_bytes;
            mem[i]->cur = cur0[i];
            cudaMemcpy(mem[i]->fld[cur0[i]], snap[i], bytes, cudaMemcpyDeviceToDevice);
            cudaMemcpy(mem[i]->d_sums_count, &cnt0[i], sizeof(long long), cudaMemcpyHostToDevice);
            cudaFree(snap[i]);
        }
        cudaDeviceSynchronize();
        return rc;
    };
    for (int i = 0; i < n; ++i) {
        const size_t bytes = mem[i]->field_cells * mem[i]->cell_bytes;
        cur0[i] = mem[i]->cur;
        if (cudaMalloc(&snap[i], bytes) != cudaSuccess) {
            cudaGetLastError();
            snap[i] = nullptr;
            err = "autotuner: no room for a state snapshot";
            return restore_and_free(WX_ENOMEM);
        }
        cudaMemcpy(snap[i], mem[i]->fld[cur0[i]], bytes, cudaMemcpyDeviceToDevice);
        cudaMemcpy(&cnt0[i], mem[i]->d_sums_count, sizeof(long long), cudaMemcpyDeviceToHost);
    }
    int deepest = 0;
    for (int i = 1; i < n; ++i)
        if (mem[i]->nz > mem[deepest]->nz) deepest = i;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    best_ms = 1e30;
    bool any = false;
    const int iters = 4;
    for (int kb : {2, 4})
        for (int ty : {2, 4, 8, 12})
            for (int st : {3, 4, 6, 8}) {
                StepCfg g;
                g.ty = ty;
                g.kb = kb;
                g.stages = st;
                g.prefetch = 0;
                g.ctas_per_sm = 1;
                int bytes = 0;
                if (!cfg_fits(mem[deepest], g, &bytes)) continue;
                const int cmax = std::min(228 * 1024 / (bytes + 1024), 2048 / (32 * (ty + 1)));
                for (int ctas = cmax; ctas >= std::max(1, cmax - 1); --ctas) {
                    g.ctas_per_sm = ctas;
                    if (!cfg_fits(mem[deepest], g, nullptr) || apply(g) != WX_OK) continue;
                    long l = 0;
                    bool ok = launch_batch(mem, n, g, status, s, &l, err) == WX_OK;  // warm-up
                    cudaEventRecord(e0, s);
                    for (int it = 0; it < iters && ok; ++it) ok = launch_batch(mem, n, g, status, s, &l, err) == WX_OK;
                    cudaEventRecord(e1, s);
                    if (!ok || cudaEventSynchronize(e1) != cudaSuccess) continue;
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    ms /= iters;
                    if (ms < best_ms) {
                        best_ms = ms;
                        best = g;
                        any = true;
                    }
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    restore_and_free(WX_OK);
    if (!any) {
        err = "autotuner: no candidate configuration ran";
        return WX_EUNSUPPORTED;
    }
    cache_store(cache, key, best, best_ms);
    return apply(best);
}

extern "C" int wx_tune(wx_ctx *c, const char *cache_path, int force, void *stream, double *best_ms) {
    if (!c) return WX_EINVAL;
    if (!c->params_set || !c->fields_loaded) {
        c->err = "wx_tune: set params and load fields first";
        return WX_ESTATE;
    }
    wx_ctx *mem[1] = {c};
    StepCfg best;
    double ms = 0;
    auto apply = [&](const StepCfg &g) {
        const int rc = apply_cfg(c, g);
        c->cfg_forced = true;
        return rc;
    };
    const int rc = tune_batch(mem, 1, c->d_status, cache_path, force, (cudaStream_t)stream, apply, best, ms, c->err);
    if (best_ms) *best_ms = ms;
    return rc;
}

extern "C" int wx_ens_tune(wx_ens *e, const char *cache_path, int force, void *stream, double *best_ms) {
    if (!e) return WX_EINVAL;
    int rc = ens_ready(e);
    if (rc != WX_OK) return rc;
    StepCfg best;
    double ms = 0;
    auto apply = [&](const StepCfg &g) { return ens_apply_cfg(e, g); };
    rc = tune_batch(e->mem.data(), (int)e->mem.size(), e->d_status, cache_path, force, (cudaStream_t)stream, apply,
                    best, ms, e->err);
    if (rc == WX_OK) e->cfg_forced = true;
    if (best_ms) *best_ms = ms;
    return rc;
}
