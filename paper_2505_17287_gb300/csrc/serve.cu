// Request loop over many independent cases on one GPU (include/ibm_serve.h).
//
// Host-only C++: worker threads, a first-in first-out admission queue, a
// stream-ordered memory pool and per-case bookkeeping. The device work of a
// case is the ordinary single-case path of ibm.h, run on the slot's stream.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/ibm.h"
#include "../../include/ibm_serve.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Slot;

// one queued or running request with its own copies of every host input
struct Req {
    int64_t id = 0;
    ibm_request r{};
    ibm_solver_opts opts{};
    bool has_opts = false;
    std::vector<double> xf, yf, zf, rhs;
    std::vector<std::vector<double>> verts;
    std::vector<std::vector<int32_t>> elems;
    std::vector<int64_t> nv, ne;
    size_t est = 0;
    bool done = false;
    ibm_result res{};
};

struct Slot {
    int index = 0;
    cudaStream_t s = nullptr;
    cudaMemPool_t pool = nullptr;
    std::thread th;
    // device bytes the running case holds, through the allocator hooks
    std::unordered_map<void *, size_t> sizes;
    size_t cur = 0, peak = 0;
    bool oom = false;
};

// allocator hooks handed to ibm_create_grid: pool allocation ordered on the
// slot stream, then a wait on that stream so the memory may also be used by
// the library's synchronous copies
void *slot_alloc(size_t bytes, void *ctx) {
    Slot *s = (Slot *)ctx;
    void *p = nullptr;
    if (cudaMallocFromPoolAsync(&p, bytes, s->pool, s->s) != cudaSuccess) {
        cudaGetLastError();
        s->oom = true;
        return nullptr;
    }
    if (cudaStreamSynchronize(s->s) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    s->sizes[p] = bytes;
    s->cur += bytes;
    s->peak = std::max(s->peak, s->cur);
    return p;
}

void slot_free(void *p, void *ctx) {
    Slot *s = (Slot *)ctx;
    auto it = s->sizes.find(p);
    if (it != s->sizes.end()) {
        s->cur -= it->second;
        s->sizes.erase(it);
    }
    cudaFreeAsync(p, s->s);
}

}  // namespace

struct ibm_server {
    ibm_server_opts opts{};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req *> queue;
    std::unordered_map<int64_t, Req *> reqs;
    std::vector<Slot *> slots;
    cudaMemPool_t pool = nullptr;
    Clock::time_point t0;
    size_t budget = 0, admitted = 0, peak_admitted = 0;
    int64_t next_id = 1, submitted = 0, completed = 0, failed = 0;
    int running = 0, peak_running = 0;
    bool stop = false;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }

    // device memory available to new cases: free memory plus what the pool
    // holds but does not use
    size_t available() {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        uint64_t reserved = 0, used = 0;
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved);
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used);
        return fr + (size_t)(reserved > used ? reserved - used : 0);
    }

    bool head_fits() {
        if (queue.empty()) return false;
        const size_t e = queue.front()->est;
        if (admitted + e > budget) return false;
        const size_t av = available();
        return av >= opts.hbm_reserve && av - opts.hbm_reserve >= e;
    }

    void worker(Slot *sl);
    void run(Req *q, Slot *sl);
};

namespace {

void set_error(ibm_result &r, ibm_status st, const char *where, const char *msg) {
    r.status = st;
    snprintf(r.error, sizeof(r.error), "%s: %s", where, msg ? msg : "");
}

}  // namespace

// one case: create, add bodies, classify, step or solve, copy results out,
// release
void ibm_server::run(Req *q, Slot *sl) {
    ibm_result &R = q->res;
    ibm_grid_desc d = q->r.grid;
    d.xf = q->xf.data();
    d.yf = q->yf.data();
    d.zf = q->zf.empty() ? nullptr : q->zf.data();
    d.stream = (void *)sl->s;
    d.alloc = slot_alloc;
    d.free = slot_free;
    d.alloc_ctx = sl;
    sl->cur = sl->peak = 0;
    sl->oom = false;
    ibm_ctx *ctx = nullptr;
    ibm_status st = ibm_create_grid(&d, &ctx);
    if (st != IBM_OK) {
        set_error(R, st, "ibm_create_grid", ibm_last_error(nullptr));
        return;
    }
    const int64_t N = (int64_t)d.nx * d.ny * (d.ndim == 3 ? d.nz : 1);
    R.cells = N;
    double *rhs_dev = nullptr, *phi_dev = nullptr;
    do {
        if (q->has_opts && (st = ibm_set_opts(ctx, &q->opts)) != IBM_OK) {
            set_error(R, st, "ibm_set_opts", ibm_last_error(ctx));
            break;
        }
        for (size_t b = 0; b < q->verts.size() && st == IBM_OK; ++b) {
            st = ibm_set_body(ctx, q->verts[b].data(), q->nv[b], q->elems[b].data(), q->ne[b]);
            if (st != IBM_OK) set_error(R, st, "ibm_set_body", ibm_last_error(ctx));
        }
        if (st != IBM_OK) break;
        if ((st = ibm_classify_cells(ctx, nullptr)) != IBM_OK) {
            set_error(R, st, "ibm_classify_cells", ibm_last_error(ctx));
            break;
        }
        if (q->r.kind == IBM_REQ_STEP) {
            st = ibm_step(ctx, q->r.nsteps, &R.step);
            R.steps = R.step.steps;
            if (st != IBM_OK) set_error(R, st, "ibm_step", ibm_last_error(ctx));
        } else {
            rhs_dev = (double *)slot_alloc(sizeof(double) * (size_t)N, sl);
            phi_dev = (double *)slot_alloc(sizeof(double) * (size_t)N, sl);
            if (!rhs_dev || !phi_dev) {
                st = IBM_ERR_OOM;
                set_error(R, st, "server", "right-hand side allocation failed");
                break;
            }
            if (cudaMemcpyAsync(rhs_dev, q->rhs.data(), sizeof(double) * (size_t)N, cudaMemcpyHostToDevice,
                                sl->s) != cudaSuccess ||
                cudaMemsetAsync(phi_dev, 0, sizeof(double) * (size_t)N, sl->s) != cudaSuccess) {
                cudaGetLastError();
                st = IBM_ERR_CUDA;
                set_error(R, st, "server", "right-hand side upload failed");
                break;
            }
            st = ibm_poisson_solve(ctx, rhs_dev, phi_dev, q->r.rtol, q->r.maxit, &R.solve);
            if (st != IBM_OK) set_error(R, st, "ibm_poisson_solve", ibm_last_error(ctx));
            if (st == IBM_OK && q->r.out_p) {
                if (cudaMemcpyAsync(q->r.out_p, phi_dev, sizeof(double) * (size_t)N, cudaMemcpyDeviceToHost,
                                    sl->s) != cudaSuccess ||
                    cudaStreamSynchronize(sl->s) != cudaSuccess) {
                    cudaGetLastError();
                    st = IBM_ERR_CUDA;
                    set_error(R, st, "server", "solution download failed");
                }
            }
        }
        // results of a completed (or converged-late) step request
        if (q->r.kind == IBM_REQ_STEP && (st == IBM_OK || st == IBM_ERR_NOT_CONVERGED)) {
            double *outs[4] = {q->r.out_u, q->r.out_v, q->r.out_w, q->r.out_p};
            const int fields[4] = {IBM_FIELD_U, IBM_FIELD_V, IBM_FIELD_W, IBM_FIELD_P};
            for (int f = 0; f < 4; ++f) {
                if (!outs[f] || (d.ndim == 2 && fields[f] == IBM_FIELD_W)) continue;   // no w in 2D
                const ibm_status s2 = ibm_get_field(ctx, fields[f], outs[f], 0, sizeof(double) * (size_t)N);
                if (s2 != IBM_OK) {
                    st = s2;
                    set_error(R, st, "ibm_get_field", ibm_last_error(ctx));
                    break;
                }
            }
        }
        if (st == IBM_OK) R.status = IBM_OK;
    } while (0);
    if (rhs_dev) slot_free(rhs_dev, sl);
    if (phi_dev) slot_free(phi_dev, sl);
    ibm_destroy(ctx);
    cudaStreamSynchronize(sl->s);
    R.bytes_peak = sl->peak;
    if (R.status == IBM_OK && st != IBM_OK) R.status = st;
}

void ibm_server::worker(Slot *sl) {
    cudaSetDevice(opts.device);
    for (;;) {
        Req *q = nullptr;
        {
            std::unique_lock<std::mutex> lk(mu);
            // re-check at least every 50 ms: free memory can change without
            // a notification (other processes, pool trimming)
            while (!stop && !head_fits()) cv_work.wait_for(lk, std::chrono::milliseconds(50));
            if (stop) return;
            q = queue.front();
            queue.pop_front();
            admitted += q->est;
            peak_admitted = std::max(peak_admitted, admitted);
            ++running;
            peak_running = std::max(peak_running, running);
            q->res.t_admit = now();
            q->res.slot = sl->index;
        }
        q->res.status = IBM_ERR_STATE;   // overwritten by run()
        run(q, sl);
        {
            std::lock_guard<std::mutex> lk(mu);
            admitted -= q->est;
            --running;
            q->res.t_done = now();
            q->done = true;
            ++completed;
            if (q->res.status != IBM_OK) ++failed;
        }
        cv_done.notify_all();
        cv_work.notify_all();
    }
}

// Upper bound on the device bytes of one case. Per cell: fields, faces,
// predictor and Poisson vectors, ghost-row scratch and the multigrid
// hierarchy of the chosen precision (coarse levels add 1/7 in 3D, 1/3 in
// 2D), the FGMRES(16) basis in the Krylov precision, and the transient
// open-area arrays of the hierarchy build; plus the body and table storage.
extern "C" size_t ibm_case_bytes(int ndim, int nx, int ny, int nz, int precision, int64_t nelems_total) {
    const double n = (double)nx * ny * (ndim == 3 ? nz : 1);
    const double coarse = ndim == 3 ? 8.0 / 7.0 : 4.0 / 3.0;
    double per_cell = 216.0;                  // FP64 fields, faces and step vectors
    per_cell += 3 * 8 * coarse;               // open areas during the hierarchy build
    if (precision == IBM_MIXED)
        per_cell += 33 * 4 + 60 * coarse + 48;  // FP32 basis, FP32 hierarchy, FP32 operator
    else
        per_cell += 33 * 8 + 90 * coarse;       // FP64 basis and hierarchy
    per_cell += 8 + 16 * 8;                   // Poisson guess history, default 8 pairs
    const double body = 256.0 * (double)nelems_total;
    return (size_t)(1.25 * (per_cell * n + body)) + ((size_t)64 << 20);
}

extern "C" ibm_status ibm_server_create(const ibm_server_opts *o, ibm_server **out) {
    if (!o || !out) return IBM_ERR_ARG;
    *out = nullptr;
    if (o->max_slots < 1 || o->max_slots > 64) return IBM_ERR_ARG;
    if (cudaSetDevice(o->device) != cudaSuccess) {
        cudaGetLastError();
        return IBM_ERR_CUDA;
    }
    ibm_server *s = new ibm_server();
    s->opts = *o;
    s->t0 = Clock::now();
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = o->device;
    if (cudaMemPoolCreate(&s->pool, &props) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return IBM_ERR_CUDA;
    }
    // keep freed memory in the pool for the next case
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        cudaMemPoolDestroy(s->pool);
        delete s;
        return IBM_ERR_CUDA;
    }
    const size_t avail = fr > o->hbm_reserve ? fr - o->hbm_reserve : 0;
    s->budget = o->hbm_budget ? std::min(o->hbm_budget, avail) : avail;
    for (int i = 0; i < o->max_slots; ++i) {
        Slot *sl = new Slot();
        sl->index = i;
        sl->pool = s->pool;
        if (cudaStreamCreateWithFlags(&sl->s, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete sl;
            ibm_server_destroy(s);
            return IBM_ERR_CUDA;
        }
        s->slots.push_back(sl);
    }
    for (Slot *sl : s->slots) sl->th = std::thread([s, sl] { s->worker(sl); });
    *out = s;
    return IBM_OK;
}

extern "C" ibm_status ibm_server_submit(ibm_server *s, const ibm_request *r, int64_t *id) {
    if (!s || !r || !id) return IBM_ERR_ARG;
    const ibm_grid_desc &g = r->grid;
    if ((g.ndim != 2 && g.ndim != 3) || g.nx < 2 || g.ny < 2 || (g.ndim == 3 && g.nz < 2) || !g.xf || !g.yf ||
        (g.ndim == 3 && !g.zf))
        return IBM_ERR_ARG;
    if (r->kind != IBM_REQ_STEP && r->kind != IBM_REQ_POISSON) return IBM_ERR_ARG;
    if (r->kind == IBM_REQ_STEP && r->nsteps < 1) return IBM_ERR_ARG;
    if (r->kind == IBM_REQ_POISSON && !r->rhs) return IBM_ERR_ARG;
    if (r->nbodies < 1 || !r->verts || !r->nverts || !r->elems || !r->nelems) return IBM_ERR_ARG;
    const int nz = g.ndim == 3 ? g.nz : 1;
    const int64_t N = (int64_t)g.nx * g.ny * nz;
    Req *q = new Req();
    q->r = *r;
    q->xf.assign(g.xf, g.xf + g.nx + 1);
    q->yf.assign(g.yf, g.yf + g.ny + 1);
    if (g.ndim == 3) q->zf.assign(g.zf, g.zf + g.nz + 1);
    if (r->opts) {
        q->opts = *r->opts;
        q->has_opts = true;
    }
    int64_t ne_total = 0;
    const int per_e = g.ndim == 3 ? 3 : 2;
    for (int b = 0; b < r->nbodies; ++b) {
        if (!r->verts[b] || !r->elems[b] || r->nverts[b] < 1 || r->nelems[b] < 1) {
            delete q;
            return IBM_ERR_ARG;
        }
        q->verts.emplace_back(r->verts[b], r->verts[b] + 3 * r->nverts[b]);
        q->elems.emplace_back(r->elems[b], r->elems[b] + per_e * r->nelems[b]);
        q->nv.push_back(r->nverts[b]);
        q->ne.push_back(r->nelems[b]);
        ne_total += r->nelems[b];
    }
    if (r->kind == IBM_REQ_POISSON) q->rhs.assign(r->rhs, r->rhs + N);
    // the copies replace every borrowed host pointer except the outputs
    q->r.grid.xf = q->r.grid.yf = q->r.grid.zf = nullptr;
    q->r.opts = nullptr;
    q->r.verts = nullptr;
    q->r.elems = nullptr;
    q->r.nverts = q->r.nelems = nullptr;
    q->r.rhs = nullptr;
    const int prec = q->has_opts ? q->opts.precision : g.precision;
    q->est = ibm_case_bytes(g.ndim, g.nx, g.ny, nz, prec, ne_total);
    if (q->has_opts && q->opts.poisson_hist > 8)   // a longer guess history than the estimate's 8 pairs
        q->est += (size_t)(1.25 * 16.0 * (q->opts.poisson_hist - 8) * (double)N);
    q->res.bytes_estimate = q->est;
    q->res.cells = N;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) {
            delete q;
            return IBM_ERR_STATE;
        }
        if (q->est > s->budget) {
            delete q;
            return IBM_ERR_OOM;
        }
        q->id = s->next_id++;
        q->res.t_submit = s->now();
        s->reqs[q->id] = q;
        s->queue.push_back(q);
        ++s->submitted;
        *id = q->id;
    }
    s->cv_work.notify_all();
    return IBM_OK;
}

extern "C" ibm_status ibm_server_wait(ibm_server *s, int64_t id, double timeout_s, ibm_result *out) {
    if (!s) return IBM_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return IBM_ERR_ARG;
    Req *q = it->second;
    auto ready = [q] { return q->done; };
    if (timeout_s < 0) s->cv_done.wait(lk, ready);
    else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) return IBM_ERR_TIMEOUT;
    if (out) *out = q->res;
    s->reqs.erase(it);
    delete q;
    return IBM_OK;
}

extern "C" ibm_status ibm_server_get_stats(ibm_server *s, ibm_server_stats *out) {
    if (!s || !out) return IBM_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->failed = s->failed;
    out->queued = (int64_t)s->queue.size();
    out->running = s->running;
    out->peak_running = s->peak_running;
    out->budget = s->budget;
    out->admitted_bytes = s->admitted;
    out->peak_admitted_bytes = s->peak_admitted;
    return IBM_OK;
}

extern "C" ibm_status ibm_server_destroy(ibm_server *s) {
    if (!s) return IBM_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        // queued requests never start; their waiters see IBM_ERR_STATE
        for (Req *q : s->queue) {
            q->res.status = IBM_ERR_STATE;
            snprintf(q->res.error, sizeof(q->res.error), "server shut down before admission");
            q->done = true;
            ++s->completed;
            ++s->failed;
        }
        s->queue.clear();
    }
    s->cv_work.notify_all();
    s->cv_done.notify_all();
    for (Slot *sl : s->slots)
        if (sl->th.joinable()) sl->th.join();
    for (Slot *sl : s->slots) {
        if (sl->s) cudaStreamDestroy(sl->s);
        delete sl;
    }
    for (auto &kv : s->reqs) delete kv.second;
    if (s->pool) cudaMemPoolDestroy(s->pool);
    delete s;
    return IBM_OK;
}

// ---------------------------------------------------------------------------
// autotuner
// ---------------------------------------------------------------------------

extern "C" ibm_status ibm_tune(const ibm_grid_desc *desc, int nbodies, const double *const *verts,
                               const int64_t *nverts, const int32_t *const *elems, const int64_t *nelems,
                               const ibm_solver_opts *cand, int ncand, int steps, int *best, double *ms_per_step) {
    if (!desc || nbodies < 1 || !verts || !nverts || !elems || !nelems || !cand || ncand < 1 || steps < 1 || !best ||
        !ms_per_step)
        return IBM_ERR_ARG;
    ibm_ctx *ctx = nullptr;
    ibm_status st = ibm_create_grid(desc, &ctx);
    if (st != IBM_OK) return st;
    const int nz = desc->ndim == 3 ? desc->nz : 1;
    const int64_t N = (int64_t)desc->nx * desc->ny * nz;
    // state fields and their sizes (doubles; the step counter is one int64)
    std::vector<std::pair<int, size_t>> fields = {{IBM_FIELD_U, N}, {IBM_FIELD_V, N}, {IBM_FIELD_P, N},
                                                  {IBM_FIELD_FACE_U, (size_t)(desc->nx + 1) * desc->ny * nz},
                                                  {IBM_FIELD_FACE_V, (size_t)desc->nx * (desc->ny + 1) * nz},
                                                  {IBM_FIELD_NOLD_U, N}, {IBM_FIELD_NOLD_V, N}};
    if (desc->ndim == 3) {
        fields.push_back({IBM_FIELD_W, N});
        fields.push_back({IBM_FIELD_FACE_W, (size_t)desc->nx * desc->ny * (nz + 1)});
        fields.push_back({IBM_FIELD_NOLD_W, N});
    }
    std::vector<std::vector<double>> saved(fields.size());
    cudaStream_t s = (cudaStream_t)desc->stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    do {
        for (int b = 0; b < nbodies && st == IBM_OK; ++b) st = ibm_set_body(ctx, verts[b], nverts[b], elems[b], nelems[b]);
        if (st != IBM_OK || (st = ibm_classify_cells(ctx, nullptr)) != IBM_OK) break;
        for (size_t f = 0; f < fields.size() && st == IBM_OK; ++f) {
            saved[f].resize(fields[f].second);
            st = ibm_get_field(ctx, fields[f].first, saved[f].data(), 0, sizeof(double) * fields[f].second);
        }
        if (st != IBM_OK) break;
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
            cudaGetLastError();
            st = IBM_ERR_CUDA;
            break;
        }
        // every candidate starts from the same state with an empty Poisson
        // guess history (pairs from an earlier candidate's solves of the same
        // steps would make the later ones look faster)
        auto restore = [&](int hist) {
            ibm_status r = IBM_OK;
            for (size_t f = 0; f < fields.size() && r == IBM_OK; ++f)
                r = ibm_set_field(ctx, fields[f].first, saved[f].data(), 0, sizeof(double) * fields[f].second);
            const int64_t zero = 0;
            if (r == IBM_OK) r = ibm_set_field(ctx, IBM_FIELD_STEP, &zero, 0, sizeof(int64_t));
            if (r == IBM_OK && hist > 0) {
                const std::vector<double> empty((size_t)(2 + hist * hist), 0.0);
                r = ibm_set_field(ctx, IBM_FIELD_P_HIST_CTL, empty.data(), 0, sizeof(double) * empty.size());
            }
            return r;
        };
        int bi = -1;
        for (int i = 0; i < ncand; ++i) {
            ms_per_step[i] = -1.0;
            if (ibm_set_opts(ctx, &cand[i]) != IBM_OK) continue;
            const int hist = cand[i].poisson_hist;
            if (restore(hist) != IBM_OK || ibm_step(ctx, 1, nullptr) != IBM_OK) continue;
            if (restore(hist) != IBM_OK) continue;
            if (cudaEventRecord(e0, s) != cudaSuccess) break;
            const ibm_status r = ibm_step(ctx, steps, nullptr);
            if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) break;
            float ms = 0.f;
            if (r != IBM_OK || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) continue;
            ms_per_step[i] = ms / steps;
            if (bi < 0 || ms_per_step[i] < ms_per_step[bi]) bi = i;
        }
        cudaGetLastError();
        if (bi < 0) {
            st = IBM_ERR_NOT_CONVERGED;
            break;
        }
        *best = bi;
    } while (0);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    ibm_destroy(ctx);
    return st;
}
