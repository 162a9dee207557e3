// bsq_server.cu -- continuous batching of simulation requests over the batch
// API (include/bsq.h): requests wait in a FIFO queue on the host, are admitted
// as slots and device memory (a byte budget) allow, advance together in one
// batch with their own adaptive dt, and leave the batch when they reach their
// end time, while later arrivals join between rounds.  Host code only; it uses
// nothing but the library's public C ABI.
#include <math.h>
#include <string.h>

#include <deque>
#include <map>
#include <new>
#include <vector>

#include "../../include/bsq.h"

namespace {

struct Request {
    long long id;
    bsq_params p;
    int bc_type[4];
    double sponge[4];
    std::vector<double> bed, eta0, P0, Q0, amp, freq, phase, dir;
    double t_end;
    size_t bytes;
    int state;  // BSQ_REQ_*
    bsq_status status;
    bsq_domain *dom;
    double t;
    long long steps;
};

}  // namespace

struct bsq_server {
    bsq_server_config cfg;
    void *stream;
    long long next_id;
    size_t used;
    std::deque<Request *> pending;
    std::vector<Request *> running;
    std::map<long long, Request *> all;
    bsq_batch *batch;
    bool dirty;  // membership changed since the batch was built
};

static void copy_in(std::vector<double> &v, const double *src, size_t n)
{
    if (src) v.assign(src, src + n);
    else v.clear();
}

static const double *ptr_or_null(const std::vector<double> &v) { return v.empty() ? nullptr : v.data(); }

extern "C" bsq_status bsq_server_create(const bsq_server_config *cfg, bsq_server **out)
{
    if (!out) return BSQ_ERR_ARG;
    *out = nullptr;
    if (!cfg || (cfg->precision != BSQ_FP32 && cfg->precision != BSQ_FP64)) return BSQ_ERR_ARG;
    bsq_server *s = new (std::nothrow) bsq_server();
    if (!s) return BSQ_ERR_OOM;
    s->cfg = *cfg;
    if (s->cfg.max_slots <= 0) s->cfg.max_slots = 64;
    if (s->cfg.steps_per_round <= 0) s->cfg.steps_per_round = 32;
    s->stream = cfg->cuda_stream;
    s->next_id = 1;
    *out = s;
    return BSQ_OK;
}

extern "C" bsq_status bsq_server_submit(bsq_server *s, const bsq_params *p, const double *bed_corners,
                                        const bsq_boundary *bnd, const double *eta0, const double *P0,
                                        const double *Q0, double t_end, long long *id)
{
    if (id) *id = 0;
    if (!s || !p || !bed_corners || !id || !(t_end > 0.0) || !isfinite(t_end)) return BSQ_ERR_ARG;
    if (p->precision != s->cfg.precision || (p->precision == BSQ_FP32 && (p->kahan != 0) != (s->cfg.kahan != 0)) ||
        p->cross_mode != BSQ_CROSS_SEQUENTIAL)
        return BSQ_ERR_ARG;
    // the batched kernels' limits: default kernel shapes, ny <= 2048, rows
    // the warp-per-row x-solver holds
    for (int q = 0; q < 8; q++)
        if (p->tune[q] != 0) return BSQ_ERR_ARG;
    const int rowmax = p->precision == BSQ_FP64 ? 3072 : 6144;
    if (p->ny > 2048 || p->nx > rowmax) return BSQ_ERR_ARG;
    const int nc = bnd ? bnd->n_comp : 0;
    const size_t bytes = bsq_domain_bytes(p, nc);
    if (bytes == 0 || (s->cfg.hbm_budget > 0 && bytes > s->cfg.hbm_budget)) return BSQ_ERR_ARG;
    Request *r = new (std::nothrow) Request();
    if (!r) return BSQ_ERR_OOM;
    r->id = s->next_id++;
    r->p = *p;
    memset(r->bc_type, 0, sizeof(r->bc_type));
    memset(r->sponge, 0, sizeof(r->sponge));
    const size_t ncell = (size_t)p->nx * p->ny;
    copy_in(r->bed, bed_corners, (size_t)(p->nx + 1) * (p->ny + 1));
    copy_in(r->eta0, eta0, ncell);
    copy_in(r->P0, P0, ncell);
    copy_in(r->Q0, Q0, ncell);
    if (bnd) {
        for (int q = 0; q < 4; q++) { r->bc_type[q] = bnd->type[q]; r->sponge[q] = bnd->sponge_width[q]; }
        if (nc > 0) {
            if (!bnd->amp || !bnd->freq || !bnd->phase || !bnd->dir) { delete r; return BSQ_ERR_ARG; }
            copy_in(r->amp, bnd->amp, nc);
            copy_in(r->freq, bnd->freq, nc);
            copy_in(r->phase, bnd->phase, nc);
            copy_in(r->dir, bnd->dir, nc);
        }
    }
    r->t_end = t_end;
    r->bytes = bytes;
    r->state = BSQ_REQ_PENDING;
    r->status = BSQ_OK;
    s->pending.push_back(r);
    s->all[r->id] = r;
    *id = r->id;
    return BSQ_OK;
}

// Create the head request's domain on the device; false if it failed (the
// request is then finished with that status).
static bool admit(bsq_server *s, Request *r)
{
    bsq_boundary b;
    memset(&b, 0, sizeof(b));
    for (int q = 0; q < 4; q++) { b.type[q] = r->bc_type[q]; b.sponge_width[q] = r->sponge[q]; }
    b.n_comp = (int)r->amp.size();
    b.amp = ptr_or_null(r->amp);
    b.freq = ptr_or_null(r->freq);
    b.phase = ptr_or_null(r->phase);
    b.dir = ptr_or_null(r->dir);
    bsq_domain *d = nullptr;
    bsq_status st = bsq_create(&r->p, r->bed.data(), &b, ptr_or_null(r->eta0), ptr_or_null(r->P0),
                               ptr_or_null(r->Q0), s->stream, &d);
    // the inputs are on the device now (or the request failed)
    std::vector<double>().swap(r->bed);
    std::vector<double>().swap(r->eta0);
    std::vector<double>().swap(r->P0);
    std::vector<double>().swap(r->Q0);
    if (st != BSQ_OK) {
        r->state = BSQ_REQ_FAILED;
        r->status = st;
        return false;
    }
    r->dom = d;
    r->state = BSQ_REQ_RUNNING;
    return true;
}

extern "C" bsq_status bsq_server_poll(bsq_server *s, int *n_running, int *n_pending)
{
    if (!s) return BSQ_ERR_ARG;
    // admission: first come, first served, while a slot and the budget allow
    while (!s->pending.empty() && (int)s->running.size() < s->cfg.max_slots) {
        Request *r = s->pending.front();
        if (s->cfg.hbm_budget > 0 && s->used + r->bytes > s->cfg.hbm_budget) break;
        s->pending.pop_front();
        if (admit(s, r)) {
            s->used += r->bytes;
            s->running.push_back(r);
            s->dirty = true;
        }
    }
    bsq_status ret = BSQ_OK;
    if (!s->running.empty()) {
        if (s->dirty) {
            // the batch is rebuilt in place (buffers and graph reused)
            std::vector<bsq_domain *> doms;
            for (Request *r : s->running) doms.push_back(r->dom);
            bsq_status st = BSQ_ERR_ARG;
            if (s->batch) {
                st = bsq_batch_reset(s->batch, doms.data(), (int)doms.size());
                if (st != BSQ_OK) {
                    bsq_batch_destroy(s->batch);
                    s->batch = nullptr;
                }
            }
            if (!s->batch) st = bsq_batch_create(doms.data(), (int)doms.size(), s->stream, &s->batch);
            if (st != BSQ_OK) return st;
            s->dirty = false;
        }
        std::vector<double> tend;
        for (Request *r : s->running) tend.push_back(r->t_end);
        std::vector<long long> done(s->running.size());
        bsq_status st = bsq_batch_advance(s->batch, tend.data(), s->cfg.steps_per_round, done.data());
        // member failures are per request; anything else fails the call
        if (st != BSQ_OK && st != BSQ_ERR_NONFINITE && st != BSQ_ERR_UNSTABLE) ret = st;
        // retire finished and failed members (their memory stays in use until released)
        std::vector<Request *> keep;
        for (Request *r : s->running) {
            double t = 0.0;
            long long n = 0;
            bsq_status rs = bsq_clock(r->dom, &t, &n);
            r->t = t;
            r->steps = n;
            const double tol = 1e-12 * fmax(1.0, fabs(r->t_end));
            if (rs != BSQ_OK) {
                r->state = BSQ_REQ_FAILED;
                r->status = rs;
                s->dirty = true;
            } else if (!(t < r->t_end - tol)) {
                r->state = BSQ_REQ_DONE;
                s->dirty = true;
            } else {
                keep.push_back(r);
            }
        }
        s->running.swap(keep);
    }
    if (n_running) *n_running = (int)s->running.size();
    if (n_pending) *n_pending = (int)s->pending.size();
    return ret;
}

extern "C" bsq_status bsq_server_request(const bsq_server *s, long long id, int *state, double *t,
                                         long long *steps, int *status)
{
    if (!s) return BSQ_ERR_ARG;
    auto it = s->all.find(id);
    if (it == s->all.end()) return BSQ_ERR_ARG;
    const Request *r = it->second;
    if (state) *state = r->state;
    if (t) *t = r->t;
    if (steps) *steps = r->steps;
    if (status) *status = (int)r->status;
    return BSQ_OK;
}

extern "C" bsq_status bsq_server_read(const bsq_server *s, long long id, int field, double *host_out)
{
    if (!s || !host_out) return BSQ_ERR_ARG;
    auto it = s->all.find(id);
    if (it == s->all.end()) return BSQ_ERR_ARG;
    const Request *r = it->second;
    if (r->state != BSQ_REQ_DONE || !r->dom) return BSQ_ERR_STATE;
    return bsq_read(r->dom, field, host_out);
}

extern "C" bsq_status bsq_server_release(bsq_server *s, long long id)
{
    if (!s) return BSQ_ERR_ARG;
    auto it = s->all.find(id);
    if (it == s->all.end()) return BSQ_ERR_ARG;
    Request *r = it->second;
    if (r->state == BSQ_REQ_PENDING || r->state == BSQ_REQ_RUNNING) return BSQ_ERR_STATE;
    if (r->dom) {
        bsq_destroy(r->dom);
        s->used -= r->bytes;
    }
    s->all.erase(it);
    delete r;
    return BSQ_OK;
}

extern "C" size_t bsq_server_bytes_in_use(const bsq_server *s) { return s ? s->used : 0; }

extern "C" void bsq_server_destroy(bsq_server *s)
{
    if (!s) return;
    bsq_batch_destroy(s->batch);
    for (auto &kv : s->all) {
        if (kv.second->dom) bsq_destroy(kv.second->dom);
        delete kv.second;
    }
    delete s;
}
