// server.cu -- continuous-batching request loop over the batch API (no counterpart in the paper,
// which relaxes one problem at a time).
//
// Jobs (a problem plus its initial particles) are submitted at any time and queued on the host.
// Each scheduling round (sph_server_poll) retires the resident jobs whose controller finished
// (DONE), ran out of iterations or failed, copying their particles back to host memory and
// emptying their instance; admits queued jobs, in arrival order, into free instances while
// their particles fit the free slots (device memory is allocated once, so admission is by
// memory); and advances every resident job together by a fixed number of steps.  Jobs of the
// two ambient dimensions live in two batches on two streams, so their steps overlap on the GPU.
// Every result is the one the job gives alone: a batch instance's arithmetic does not depend
// on the other instances.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <string>
#include <vector>

#include "../../include/sphmesh.h"
#include "sph_internal.cuh"

namespace {

sph_status sfail(sph_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    sph::set_last_error(buf);
    return s;
}

struct Job {
    sph_domain_desc dom;
    sph_sizing_desc siz;
    sph_params prm;
    std::vector<double> x, h;
    std::vector<int32_t> g;
    int64_t n = 0, max_iters = 0;
    int32_t state = SPH_JOB_QUEUED;
    int lane = -1, side = 0;         // instance and batch (0: 2D, 1: 3D) while resident
    sph_job_info info;
    std::vector<double> xo, ho;       // results
    std::vector<int32_t> go;
    bool sampled = false;             // particles drawn on the device at admission (Sec. 3.6)
    uint64_t seed = 0;
    std::vector<int64_t> counts;      // per feature, fixed at submission
};

struct Side {
    sph_batch* b = nullptr;
    int64_t slot_cap = 0, slots_used = 0;
    std::vector<int64_t> lane_job;   // job id per instance, -1: free
};

int64_t slots_of(int64_t n) { return (n + sph::CHUNK - 1) / sph::CHUNK * sph::CHUNK; }

// a small valid problem for instances that hold no job
void placeholder(int dim, int precision, sph_domain_desc* d, sph_sizing_desc* z, sph_params* p) {
    std::memset(d, 0, sizeof *d);
    std::memset(z, 0, sizeof *z);
    d->dim = dim;
    d->base = 0;
    for (int a = 0; a < 3; ++a) {
        d->bbox_lo[a] = 0.0;
        d->bbox_hi[a] = a < dim ? 1.0 : 0.0;
    }
    d->n_features = 1;
    d->features[0].kind = SPH_FEAT_VOLUME;
    d->features[0].dim = dim;
    z->kind = 0;
    z->a = z->lo = z->hi = 0.25;
    sph_params_default(p);
    p->precision = precision;
}

double now_s(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct sph_server {
    sph_server_config cfg;
    Side side[2];
    cudaStream_t samp = nullptr;      // the sampling of descriptor-only jobs
    std::map<int64_t, Job> jobs;
    std::deque<int64_t> queue;
    int64_t next_id = 1;
    std::chrono::steady_clock::time_point t0;
    sph_server_stats stats;
};

namespace {

void server_free(sph_server* s) {
    for (Side& d : s->side)
        if (d.b) sph_batch_destroy(d.b);
    if (s->samp) cudaStreamDestroy(s->samp);
}

// copies a finished job's particles to host memory and empties its instance
sph_status retire(sph_server* s, Job& j, int64_t id, int32_t state, const sph_report& r) {
    Side& d = s->side[j.side];
    j.xo.assign((size_t)j.n * 3, 0.0);
    j.go.assign((size_t)j.n, 0);
    j.ho.assign((size_t)j.n, 0.0);
    int64_t got = 0;
    sph_status st = sph_batch_positions(d.b, j.lane, j.xo.data(), j.go.data(), nullptr, j.ho.data(), j.n, &got);
    if (st != SPH_OK) return st;
    st = sph_batch_set_state(d.b, j.lane, 0, nullptr, nullptr, nullptr, nullptr);
    if (st != SPH_OK) return st;
    d.lane_job[j.lane] = -1;
    d.slots_used -= slots_of(j.n);
    j.state = state;
    j.info.state = state;
    j.info.iterations = r.iteration;
    j.info.phase = r.phase;
    j.info.E_sys = r.E_sys;
    j.info.escapes = r.escapes;
    j.info.status_word = r.status;
    j.info.t_finish = now_s(s->t0);
    j.lane = -1;
    j.x.clear();
    j.x.shrink_to_fit();
    j.h.clear();
    j.h.shrink_to_fit();
    j.g.clear();
    j.g.shrink_to_fit();
    s->stats.finished += 1;
    (void)id;
    return SPH_OK;
}

sph_status admit(sph_server* s, Job& j, int lane) {
    Side& d = s->side[j.side];
    if (j.sampled && j.x.empty()) {
        j.x.resize((size_t)j.n * 3);
        j.g.resize((size_t)j.n);
        sph_status st = sph_sample_particles(&j.dom, &j.siz, j.seed, j.counts.data(), s->samp, j.x.data(), j.g.data());
        if (st != SPH_OK) return st;
    }
    sph_status st = sph_batch_set_problem(d.b, lane, &j.dom, &j.siz, &j.prm);
    if (st != SPH_OK) return st;
    st = sph_batch_set_state(d.b, lane, j.n, j.x.data(), j.g.data(), nullptr, j.h.empty() ? nullptr : j.h.data());
    if (st != SPH_OK) return st;
    d.slots_used += slots_of(j.n);
    j.lane = lane;
    j.state = SPH_JOB_RUNNING;
    j.info.state = SPH_JOB_RUNNING;
    j.info.t_admit = now_s(s->t0);
    return SPH_OK;
}

}  // namespace

#pragma GCC visibility push(default)
extern "C" {

sph_status sph_server_create(const sph_server_config* cfg, sph_server** out) {
    if (!cfg || !out) return sfail(SPH_E_INVALID, "server_create: NULL argument");
    *out = nullptr;
    if (cfg->precision != 32 && cfg->precision != 64) return sfail(SPH_E_INVALID, "server: precision must be 32 or 64");
    if (cfg->max_jobs < 1 || cfg->max_jobs > SPH_MAX_INSTANCES)
        return sfail(SPH_E_INVALID, "server: max_jobs must be in [1, %d]", SPH_MAX_INSTANCES);
    if (cfg->slot_capacity[0] < -1 || cfg->slot_capacity[1] < -1 || (cfg->slot_capacity[0] == 0 && cfg->slot_capacity[1] == 0))
        return sfail(SPH_E_INVALID, "server: need a slot capacity for at least one dimension");
    if (cfg->steps_per_poll < 1) return sfail(SPH_E_INVALID, "server: steps_per_poll must be positive");
    sph_server_config c = *cfg;
    const int autos = (c.slot_capacity[0] < 0) + (c.slot_capacity[1] < 0);
    if (autos > 0) {
        if (!(c.hbm_fraction > 0.0 && c.hbm_fraction < 1.0)) return sfail(SPH_E_INVALID, "server: hbm_fraction must be in (0, 1)");
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return sfail(SPH_E_CUDA, "server: cudaMemGetInfo failed");
        for (int k = 0; k < 2; ++k)
            if (c.slot_capacity[k] < 0) {
                int64_t per = 0;
                sph_status st = sph_batch_slot_bytes(k == 0 ? 2 : 3, c.precision, &per);
                if (st != SPH_OK) return st;
                c.slot_capacity[k] = (int64_t)((double)fr * c.hbm_fraction / autos / (double)per);
                c.slot_capacity[k] = std::min<int64_t>(c.slot_capacity[k], ((int64_t)1 << 31) / 16);
                if (c.slot_capacity[k] < sph::CHUNK) return sfail(SPH_E_NOMEM, "server: no device memory for %dD jobs", k + 2);
            }
    }
    sph_server* s = new sph_server();
    s->cfg = c;
    if (cudaStreamCreateWithFlags(&s->samp, cudaStreamNonBlocking) != cudaSuccess) {
        delete s;
        return sfail(SPH_E_CUDA, "server: cudaStreamCreateWithFlags failed");
    }
    std::memset(&s->stats, 0, sizeof s->stats);
    s->t0 = std::chrono::steady_clock::now();
    for (int k = 0; k < 2; ++k) {
        if (c.slot_capacity[k] == 0) continue;
        const int NI = c.max_jobs;
        std::vector<sph_domain_desc> doms(NI);
        std::vector<sph_sizing_desc> sizs(NI);
        std::vector<sph_params> prms(NI);
        std::vector<int64_t> caps(NI);
        const int64_t per = (c.slot_capacity[k] + NI - 1) / NI;
        for (int i = 0; i < NI; ++i) {
            placeholder(k == 0 ? 2 : 3, c.precision, &doms[i], &sizs[i], &prms[i]);
            caps[i] = per;
        }
        sph_status st = sph_batch_create(NI, doms.data(), sizs.data(), prms.data(), caps.data(), nullptr, &s->side[k].b);
        if (st != SPH_OK) {
            server_free(s);
            delete s;
            return st;
        }
        int64_t cap = 0;
        sph_batch_size(s->side[k].b, nullptr, nullptr, &cap);
        s->side[k].slot_cap = cap;
        s->side[k].lane_job.assign(NI, -1);
    }
    *out = s;
    return SPH_OK;
}

sph_status sph_server_submit(sph_server* s, const sph_domain_desc* dom, const sph_sizing_desc* siz,
                             const sph_params* prm, int64_t n, const double* x, const int32_t* group, const double* h,
                             int64_t max_iters, int64_t* job_id) {
    if (!s || !dom || !siz || !prm || !job_id) return sfail(SPH_E_INVALID, "submit: NULL argument");
    if (dom->dim != 2 && dom->dim != 3) return sfail(SPH_E_INVALID, "submit: dim must be 2 or 3");
    const int k = dom->dim == 2 ? 0 : 1;
    if (!s->side[k].b) return sfail(SPH_E_INVALID, "submit: the server holds no %dD capacity", dom->dim);
    if (prm->precision != s->cfg.precision) return sfail(SPH_E_INVALID, "submit: precision differs from the server's");
    if (n < 1 || !x || !group) return sfail(SPH_E_INVALID, "submit: need n >= 1 particles with x and group");
    if (slots_of(n) > s->side[k].slot_cap)
        return sfail(SPH_E_INVALID, "submit: %lld particles never fit the %lld slots of the server", (long long)n,
                     (long long)s->side[k].slot_cap);
    if (max_iters < 0) return sfail(SPH_E_INVALID, "submit: max_iters < 0");
    Job j;
    j.dom = *dom;
    j.siz = *siz;
    j.prm = *prm;
    j.n = n;
    j.max_iters = max_iters;
    j.side = k;
    j.x.assign(x, x + n * 3);
    j.g.assign(group, group + n);
    if (h) j.h.assign(h, h + n);
    std::memset(&j.info, 0, sizeof j.info);
    j.info.state = SPH_JOB_QUEUED;
    j.info.n = n;
    j.info.dim = dom->dim;
    j.info.t_submit = now_s(s->t0);
    const int64_t id = s->next_id++;
    s->jobs.emplace(id, std::move(j));
    s->queue.push_back(id);
    s->stats.submitted += 1;
    *job_id = id;
    return SPH_OK;
}

sph_status sph_server_submit_sampled(sph_server* s, const sph_domain_desc* dom, const sph_sizing_desc* siz,
                                     const sph_params* prm, uint64_t seed, int64_t max_iters, int64_t* job_id) {
    if (!s || !dom || !siz || !prm || !job_id) return sfail(SPH_E_INVALID, "submit: NULL argument");
    if (dom->dim != 2 && dom->dim != 3) return sfail(SPH_E_INVALID, "submit: dim must be 2 or 3");
    if (dom->n_features < 1 || dom->n_features > SPH_MAX_FEATURES) return sfail(SPH_E_INVALID, "submit: n_features out of range");
    const int k = dom->dim == 2 ? 0 : 1;
    if (!s->side[k].b) return sfail(SPH_E_INVALID, "submit: the server holds no %dD capacity", dom->dim);
    if (prm->precision != s->cfg.precision) return sfail(SPH_E_INVALID, "submit: precision differs from the server's");
    if (max_iters < 0) return sfail(SPH_E_INVALID, "submit: max_iters < 0");
    std::vector<int64_t> counts(dom->n_features);
    sph_status st = sph_feature_counts(dom, siz, s->samp, nullptr, counts.data());
    if (st != SPH_OK) return st;
    int64_t n = 0;
    for (int64_t c : counts) n += c;
    if (n < 1) return sfail(SPH_E_INVALID, "submit: the problem holds no particle");
    if (slots_of(n) > s->side[k].slot_cap)
        return sfail(SPH_E_INVALID, "submit: %lld particles never fit the %lld slots of the server", (long long)n,
                     (long long)s->side[k].slot_cap);
    Job j;
    j.dom = *dom;
    j.siz = *siz;
    j.prm = *prm;
    j.n = n;
    j.max_iters = max_iters;
    j.side = k;
    j.sampled = true;
    j.seed = seed;
    j.counts = std::move(counts);
    std::memset(&j.info, 0, sizeof j.info);
    j.info.state = SPH_JOB_QUEUED;
    j.info.n = n;
    j.info.dim = dom->dim;
    j.info.t_submit = now_s(s->t0);
    const int64_t id = s->next_id++;
    s->jobs.emplace(id, std::move(j));
    s->queue.push_back(id);
    s->stats.submitted += 1;
    *job_id = id;
    return SPH_OK;
}

sph_status sph_server_poll(sph_server* s, sph_server_stats* stats_out) {
    if (!s) return sfail(SPH_E_INVALID, "poll: NULL handle");
    // 1. retire finished jobs
    for (int k = 0; k < 2; ++k) {
        Side& d = s->side[k];
        if (!d.b) continue;
        const int NI = s->cfg.max_jobs;
        bool any = false;
        for (int i = 0; i < NI; ++i) any = any || d.lane_job[i] >= 0;
        if (!any) continue;
        std::vector<sph_report> rep(NI);
        sph_status st = sph_batch_reports(d.b, rep.data(), NI);
        if (st != SPH_OK) return st;
        for (int i = 0; i < NI; ++i) {
            const int64_t id = d.lane_job[i];
            if (id < 0) continue;
            Job& j = s->jobs.at(id);
            const sph_report& r = rep[i];
            int32_t state = 0;
            if (r.status & (sph::ST_NONFINITE | sph::ST_OUTSIDE_GRID)) state = SPH_JOB_FAILED;
            else if (r.phase == SPH_DONE) state = SPH_JOB_DONE;
            else if (r.iteration >= j.max_iters) state = SPH_JOB_NOT_CONVERGED;
            if (state) {
                st = retire(s, j, id, state, r);
                if (st != SPH_OK) return st;
            }
        }
    }
    // 2. admit queued jobs in arrival order while an instance and room are free
    for (auto it = s->queue.begin(); it != s->queue.end();) {
        Job& j = s->jobs.at(*it);
        Side& d = s->side[j.side];
        int lane = -1;
        for (int i = 0; i < (int)d.lane_job.size() && lane < 0; ++i)
            if (d.lane_job[i] < 0) lane = i;
        if (lane < 0 || d.slots_used + slots_of(j.n) > d.slot_cap) {
            ++it;
            continue;
        }
        sph_status st = admit(s, j, lane);
        if (st == SPH_E_NOMEM) {   // cell arrays did not fit: try again after retirements
            ++it;
            continue;
        }
        if (st != SPH_OK) {
            j.state = SPH_JOB_FAILED;
            j.info.state = SPH_JOB_FAILED;
            j.info.t_finish = now_s(s->t0);
            s->stats.finished += 1;
            it = s->queue.erase(it);
            continue;
        }
        d.lane_job[lane] = *it;
        it = s->queue.erase(it);
    }
    // 3. advance every resident job
    int64_t running = 0, particles = 0;
    for (int k = 0; k < 2; ++k) {
        Side& d = s->side[k];
        if (!d.b) continue;
        int64_t here = 0;
        for (int64_t id : d.lane_job)
            if (id >= 0) {
                ++here;
                particles += s->jobs.at(id).n;
            }
        running += here;
        if (here > 0) {
            sph_status st = sph_batch_step(d.b, s->cfg.steps_per_poll);
            if (st != SPH_OK) return st;
        }
    }
    for (int k = 0; k < 2; ++k)
        if (s->side[k].b) {
            // a job whose status word is set is retired as failed in the next round
            sph_status st = sph_batch_sync(s->side[k].b);
            if (st != SPH_OK && st != SPH_E_DIVERGED && st != SPH_E_OVERFLOW) return st;
        }
    s->stats.rounds += 1;
    s->stats.particle_steps += (double)particles * s->cfg.steps_per_poll;
    s->stats.running = running;
    s->stats.queued = (int64_t)s->queue.size();
    if (stats_out) *stats_out = s->stats;
    return SPH_OK;
}

sph_status sph_server_drain(sph_server* s, int64_t max_rounds, sph_server_stats* stats_out) {
    if (!s) return sfail(SPH_E_INVALID, "drain: NULL handle");
    for (int64_t r = 0; r < max_rounds; ++r) {
        sph_status st = sph_server_poll(s, stats_out);
        if (st != SPH_OK) return st;
        if (s->stats.running == 0 && s->stats.queued == 0) {
            // the last round may have retired the final jobs; one more pass retires nothing
            return SPH_OK;
        }
    }
    return sfail(SPH_E_NOT_CONVERGED, "drain: work left after %lld rounds", (long long)max_rounds);
}

sph_status sph_server_job(sph_server* s, int64_t job_id, sph_job_info* info, double* x_out, int32_t* group_out,
                          double* h_out, int64_t capacity) {
    if (!s || !info) return sfail(SPH_E_INVALID, "job: NULL argument");
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return sfail(SPH_E_INVALID, "job: unknown id %lld", (long long)job_id);
    const Job& j = it->second;
    *info = j.info;
    const bool finished = j.state == SPH_JOB_DONE || j.state == SPH_JOB_NOT_CONVERGED || j.state == SPH_JOB_FAILED;
    if ((x_out || group_out || h_out) && finished && !j.xo.empty()) {
        if (capacity < j.n) return sfail(SPH_E_INVALID, "job: capacity %lld < n %lld", (long long)capacity, (long long)j.n);
        if (x_out) std::memcpy(x_out, j.xo.data(), sizeof(double) * 3 * (size_t)j.n);
        if (group_out) std::memcpy(group_out, j.go.data(), sizeof(int32_t) * (size_t)j.n);
        if (h_out) std::memcpy(h_out, j.ho.data(), sizeof(double) * (size_t)j.n);
    }
    return SPH_OK;
}

sph_status sph_server_release(sph_server* s, int64_t job_id) {
    if (!s) return sfail(SPH_E_INVALID, "release: NULL handle");
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return sfail(SPH_E_INVALID, "release: unknown id %lld", (long long)job_id);
    const int32_t st = it->second.state;
    if (st == SPH_JOB_QUEUED || st == SPH_JOB_RUNNING) return sfail(SPH_E_INVALID, "release: job %lld is not finished", (long long)job_id);
    s->jobs.erase(it);
    return SPH_OK;
}

void sph_server_destroy(sph_server* s) {
    if (!s) return;
    server_free(s);
    delete s;
}

}  // extern "C"
#pragma GCC visibility pop
