// ohm_server.cpp -- continuous-batching solve service (include/ohm_server.h).
//
// Host runtime only: every arithmetic step runs in the batched hierarchies of libohm
// (ohm_cn_step_batch).  One mutex guards the queue, the batch table and the budget; device
// copies, steps and hierarchy creation run outside it, on each batch's own stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "ohm.h"
#include "ohm_server.h"

namespace {

constexpr int B3C = 3 * 512;  // doubles per block of B
constexpr int B1C = 512;      // doubles per block of eta

struct Req {
    int64_t id = 0;
    std::string key;
    int32_t base_cells[3];
    double dx0 = 0;
    int32_t nlevels = 0;
    int64_t nblocks = 0;
    std::vector<int32_t> lijk;
    std::vector<int64_t> lev_off, lev_n;  // per level: first block and count (one instance)
    std::vector<double> B, eta;
    double dt = 0;
    int nsteps = 0;
    double *out = nullptr;
    // progress
    int steps_done = 0;
    ohm_request_result res{};
    bool done = false;
};

struct Batch {
    std::string key;
    int K = 0;
    ohm_hier *h = nullptr;
    double *Bd = nullptr, *etad = nullptr;
    double *pin = nullptr;  // pinned staging of one instance (B then eta)
    cudaStream_t s = nullptr;
    int64_t bytes = 0;
    bool busy = false;
    double last_used = 0;
    std::vector<Req *> slot;
    // structure of one instance
    std::vector<int64_t> lev_off, lev_n;
    int64_t nb = 0;
};

}  // namespace

struct ohm_server {
    ohm_server_desc d{};
    int device = 0;
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req *> queue;
    std::map<int64_t, std::unique_ptr<Req>> reqs;
    std::list<std::unique_ptr<Batch>> batches;
    std::map<std::pair<std::string, int>, int64_t> bytes_cache;
    int64_t next_id = 1;
    int64_t resident = 0;
    bool stopping = false;
    std::vector<std::thread> workers;
    ohm_server_stats st{};
    double active_sum = 0;
    int64_t launches_freed = 0;  // launches of batches already destroyed

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

ohm_hier_desc structure_desc(const ohm_server *S, const Req *r, int K, void *stream) {
    ohm_hier_desc d{};
    for (int a = 0; a < 3; a++) d.base_cells[a] = r->base_cells[a];
    d.dx0 = r->dx0;
    d.nlevels = r->nlevels;
    d.nblocks = r->nblocks;
    d.block_lijk = r->lijk.data();
    d.lambda = S->d.lambda;
    d.precision = S->d.precision;
    d.nu_pre = S->d.nu_pre;
    d.nu_post = S->d.nu_post;
    d.n_coarse = S->d.n_coarse;
    d.max_outer = S->d.max_outer;
    d.krylov = S->d.krylov;
    d.inner_tol = 0;
    d.n_instances = K;
    d.use_graphs = S->d.use_graphs;
    d.stream = stream;
    d.omega = S->d.omega;
    d.nu_coarse_pre = S->d.nu_coarse_pre;
    d.nu_coarse_post = S->d.nu_coarse_post;
    return d;
}

// device bytes of a batch of K instances of r's class (hierarchy + B + eta); called with mu held
int64_t batch_bytes(ohm_server *S, const Req *r, int K) {
    auto it = S->bytes_cache.find({r->key, K});
    if (it != S->bytes_cache.end()) return it->second;
    ohm_hier_desc d = structure_desc(S, r, K, nullptr);
    int64_t b = 0;
    if (ohm_hierarchy_bytes(&d, &b) != OHM_OK) b = -1;
    else b += (int64_t)K * r->nblocks * (B3C + B1C) * 8;
    S->bytes_cache[{r->key, K}] = b;
    return b;
}

void free_batch(Batch *b, int64_t *launches = nullptr) {
    if (b->h && launches) *launches += ohm_launch_count(b->h);
    if (b->h) ohm_destroy(b->h);
    if (b->Bd) cudaFree(b->Bd);
    if (b->etad) cudaFree(b->etad);
    if (b->pin) cudaFreeHost(b->pin);
    if (b->s) cudaStreamDestroy(b->s);
    b->h = nullptr;
    b->Bd = b->etad = b->pin = nullptr;
    b->s = nullptr;
}

int create_batch(ohm_server *S, const Req *r, Batch *b) {
    b->slot.assign(b->K, nullptr);
    b->lev_off = r->lev_off;
    b->lev_n = r->lev_n;
    b->nb = r->nblocks;
    if (cudaStreamCreateWithFlags(&b->s, cudaStreamNonBlocking) != cudaSuccess) return OHM_ERR_CUDA;
    const size_t nB = (size_t)b->K * r->nblocks * B3C, nE = (size_t)b->K * r->nblocks * B1C;
    if (cudaMalloc(&b->Bd, nB * 8) != cudaSuccess || cudaMalloc(&b->etad, nE * 8) != cudaSuccess ||
        cudaMallocHost(&b->pin, (size_t)r->nblocks * (B3C + B1C) * 8) != cudaSuccess) {
        cudaGetLastError();
        return OHM_ERR_OOM;
    }
    // unused slots hold zero fields with eta = 1 (valid, never stepped)
    if (cudaMemsetAsync(b->Bd, 0, nB * 8, b->s) != cudaSuccess) return OHM_ERR_CUDA;
    std::vector<double> ones(std::min<size_t>(nE, (size_t)1 << 20), 1.0);
    for (size_t o = 0; o < nE; o += ones.size()) {
        const size_t n = std::min(ones.size(), nE - o);
        if (cudaMemcpyAsync(b->etad + o, ones.data(), n * 8, cudaMemcpyHostToDevice, b->s) != cudaSuccess) return OHM_ERR_CUDA;
        if (cudaStreamSynchronize(b->s) != cudaSuccess) return OHM_ERR_CUDA;
    }
    ohm_hier_desc d = structure_desc(S, r, b->K, b->s);
    int st = ohm_create_hierarchy(&d, &b->h);
    if (st) return st;
    return ohm_set_eta(b->h, b->etad);
}

// copies between one instance's host arrays (level-sorted blocks) and slot q of a batch
// (level by level, the K instances' blocks of that level one after another)
int copy_in(Batch *b, int q, const Req *r) {
    memcpy(b->pin, r->B.data(), r->B.size() * 8);
    memcpy(b->pin + r->B.size(), r->eta.data(), r->eta.size() * 8);
    for (size_t l = 0; l < b->lev_n.size(); l++) {
        const int64_t n = b->lev_n[l], src = b->lev_off[l], dst = (int64_t)b->K * b->lev_off[l] + (int64_t)q * n;
        if (cudaMemcpyAsync(b->Bd + dst * B3C, b->pin + src * B3C, n * B3C * 8, cudaMemcpyHostToDevice, b->s) ||
            cudaMemcpyAsync(b->etad + dst * B1C, b->pin + r->B.size() + src * B1C, n * B1C * 8, cudaMemcpyHostToDevice, b->s))
            return OHM_ERR_CUDA;
    }
    return cudaStreamSynchronize(b->s) == cudaSuccess ? OHM_OK : OHM_ERR_CUDA;
}

int copy_out(Batch *b, int q, Req *r) {
    for (size_t l = 0; l < b->lev_n.size(); l++) {
        const int64_t n = b->lev_n[l], dst = b->lev_off[l], src = (int64_t)b->K * b->lev_off[l] + (int64_t)q * n;
        if (cudaMemcpyAsync(b->pin + dst * B3C, b->Bd + src * B3C, n * B3C * 8, cudaMemcpyDeviceToHost, b->s)) return OHM_ERR_CUDA;
    }
    if (cudaStreamSynchronize(b->s) != cudaSuccess) return OHM_ERR_CUDA;
    memcpy(r->out, b->pin, (size_t)r->nblocks * B3C * 8);
    return OHM_OK;
}

void finish(ohm_server *S, Req *r, int status) {  // mu held
    std::vector<double>().swap(r->B);  // inputs are no longer needed
    std::vector<double>().swap(r->eta);
    r->res.status = status;
    r->res.t_done = S->now();
    r->done = true;
    S->st.requests_done++;
    S->cv_done.notify_all();
}

// Steps one batch until it has no active slot and no queued request of its class.
void run_batch(ohm_server *S, Batch *b, std::unique_lock<std::mutex> &lk) {
    std::vector<double> dts(b->K, 1.0);
    std::vector<uint8_t> active(b->K, 0);
    std::vector<ohm_step_stats> stats(b->K);
    for (;;) {
        // admission: queued requests of this class into free slots, oldest first
        std::vector<int> fresh;
        for (int q = 0; q < b->K; q++) {
            if (b->slot[q]) continue;
            auto it = std::find_if(S->queue.begin(), S->queue.end(), [&](Req *r) { return r->key == b->key; });
            if (it == S->queue.end()) break;
            b->slot[q] = *it;
            S->queue.erase(it);
            b->slot[q]->res.t_start = S->now();
            b->slot[q]->res.slot = q;
            fresh.push_back(q);
        }
        int nact = 0;
        for (int q = 0; q < b->K; q++) nact += b->slot[q] != nullptr;
        if (nact == 0) return;
        lk.unlock();
        int st = OHM_OK;
        for (int q : fresh)
            if (st == OHM_OK) st = copy_in(b, q, b->slot[q]);
        if (st == OHM_OK && !fresh.empty()) st = ohm_set_eta(b->h, b->etad);
        for (int q = 0; q < b->K; q++) {
            active[q] = b->slot[q] != nullptr;
            if (active[q]) dts[q] = b->slot[q]->dt;
        }
        if (st == OHM_OK) {
            const int s2 = ohm_cn_step_batch(b->h, b->Bd, dts.data(), S->d.tol, active.data(), stats.data());
            if (s2 != OHM_OK && s2 != OHM_ERR_NOT_CONVERGED && s2 != OHM_ERR_NONFINITE) st = s2;
        }
        // finished slots: copy out before taking the lock
        std::vector<std::pair<int, int>> ended;  // slot, status
        for (int q = 0; q < b->K; q++) {
            Req *r = b->slot[q];
            if (!r) continue;
            int rs = OHM_OK;
            if (st != OHM_OK) rs = st;
            else {
                r->res.cycles += stats[q].cycles;
                r->res.rel_l2 = stats[q].rel_l2;
                r->steps_done++;
                if (!stats[q].converged) rs = std::isfinite(stats[q].rel_l2) ? OHM_ERR_NOT_CONVERGED : OHM_ERR_NONFINITE;
            }
            if (rs != OHM_OK || r->steps_done >= r->nsteps) {
                if (st == OHM_OK && copy_out(b, q, r) != OHM_OK) rs = OHM_ERR_CUDA;
                ended.push_back({q, rs});
            }
        }
        lk.lock();
        S->st.steps_run++;
        S->active_sum += nact;
        for (auto &e : ended) {
            finish(S, b->slot[e.first], e.second);
            b->slot[e.first] = nullptr;
        }
    }
}

// the oldest queued request that no busy batch with a free slot will admit at its next step
Req *pick(ohm_server *S) {
    for (Req *r : S->queue) {
        bool served = false;
        for (auto &b : S->batches)
            if (b->busy && b->key == r->key &&
                std::count(b->slot.begin(), b->slot.end(), nullptr) > 0)
                served = true;
        if (!served) return r;
    }
    return nullptr;
}

void worker(ohm_server *S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        Req *r = nullptr;
        S->cv_work.wait(lk, [&] { return (r = pick(S)) != nullptr || (S->stopping && S->queue.empty()); });
        if (!r) return;
        // an idle resident batch of the class, else a new one within the budget
        Batch *b = nullptr;
        for (auto &x : S->batches)
            if (!x->busy && x->key == r->key) b = x.get();
        if (!b) {
            int K = S->d.max_batch;
            int64_t need = batch_bytes(S, r, K);
            while (K > 1 && (need < 0 || need > S->d.hbm_budget_bytes)) {
                K = (K + 1) / 2;
                need = batch_bytes(S, r, K);
            }
            // evict idle batches, least recently used first, until the new one fits
            while (S->resident + need > S->d.hbm_budget_bytes) {
                Batch *victim = nullptr;
                for (auto &x : S->batches)
                    if (!x->busy && (!victim || x->last_used < victim->last_used)) victim = x.get();
                if (!victim) break;
                S->resident -= victim->bytes;
                S->st.batches_evicted++;
                std::unique_ptr<Batch> owned;
                for (auto it = S->batches.begin(); it != S->batches.end(); ++it)
                    if (it->get() == victim) {
                        owned = std::move(*it);
                        S->batches.erase(it);
                        break;
                    }
                lk.unlock();
                int64_t n = 0;
                free_batch(owned.get(), &n);
                lk.lock();
                S->launches_freed += n;
            }
            if (S->resident + need > S->d.hbm_budget_bytes) {
                // the running batches hold the memory: wait for one to go idle
                S->cv_work.wait(lk);
                continue;
            }
            auto nb = std::make_unique<Batch>();
            nb->key = r->key;
            nb->K = K;
            nb->bytes = need;
            nb->busy = true;
            b = nb.get();
            S->resident += need;
            S->st.batches_created++;
            S->st.bytes_resident_max = std::max(S->st.bytes_resident_max, S->resident);
            S->batches.push_back(std::move(nb));
            lk.unlock();
            const int st = create_batch(S, r, b);
            lk.lock();
            if (st != OHM_OK) {
                // fail this class's queued requests rather than retrying forever
                for (auto it = S->queue.begin(); it != S->queue.end();) {
                    if ((*it)->key == b->key) {
                        finish(S, *it, st);
                        it = S->queue.erase(it);
                    } else
                        ++it;
                }
                S->resident -= b->bytes;
                for (auto it = S->batches.begin(); it != S->batches.end(); ++it)
                    if (it->get() == b) {
                        lk.unlock();
                        free_batch(b);
                        lk.lock();
                        S->batches.erase(it);
                        break;
                    }
                S->cv_work.notify_all();
                continue;
            }
        } else {
            b->busy = true;
        }
        run_batch(S, b, lk);
        b->busy = false;
        b->last_used = S->now();
        S->cv_work.notify_all();
    }
}

std::string class_key(const ohm_request *r) {
    std::string k;
    k.append((const char *)r->base_cells, sizeof(r->base_cells));
    k.append((const char *)&r->dx0, sizeof(double));
    k.append((const char *)&r->nlevels, sizeof(int32_t));
    k.append((const char *)r->block_lijk, (size_t)r->nblocks * 4 * sizeof(int32_t));
    return k;
}

}  // namespace

extern "C" {

int ohm_server_create(const ohm_server_desc *d, ohm_server **out) {
    if (!d || !out) return OHM_ERR_INVALID;
    *out = nullptr;
    if (d->hbm_budget_bytes <= 0 || d->max_batch < 1 || d->max_batch > 4096 || d->n_workers < 1 || d->n_workers > 64 ||
        (d->precision != OHM_FP64 && d->precision != OHM_MIXED && d->precision != OHM_MIXED_FF) || !(d->lambda > 0 && d->lambda <= 1) || !(d->tol >= 0) ||
        d->nu_pre < 0 || d->nu_post < 0 || d->n_coarse < 1 || d->max_outer < 1 || d->krylov < 0 || d->krylov > 11 ||
        (d->krylov > 0 && d->precision == OHM_FP64) || !(d->omega == 0 || (d->omega > 0 && d->omega < 2)) ||
        d->nu_coarse_pre < 0 || d->nu_coarse_post < 0)
        return OHM_ERR_INVALID;
    ohm_server *S = new ohm_server();
    S->d = *d;
    S->t0 = std::chrono::steady_clock::now();
    if (cudaGetDevice(&S->device) != cudaSuccess) {
        cudaGetLastError();
        delete S;
        return OHM_ERR_CUDA;
    }
    for (int i = 0; i < d->n_workers; i++) S->workers.emplace_back(worker, S);
    *out = S;
    return OHM_OK;
}

int ohm_server_submit(ohm_server *S, const ohm_request *r, int64_t *id) {
    if (!S || !r || !id || !r->block_lijk || !r->B || !r->eta || !r->B_out || r->nblocks <= 0 || r->nlevels < 1 ||
        !(r->dt > 0) || !std::isfinite(r->dt) || r->nsteps < 1)
        return OHM_ERR_INVALID;
    auto q = std::make_unique<Req>();
    q->key = class_key(r);
    for (int a = 0; a < 3; a++) q->base_cells[a] = r->base_cells[a];
    q->dx0 = r->dx0;
    q->nlevels = r->nlevels;
    q->nblocks = r->nblocks;
    q->lijk.assign(r->block_lijk, r->block_lijk + 4 * r->nblocks);
    q->lev_off.assign(r->nlevels, 0);
    q->lev_n.assign(r->nlevels, 0);
    for (int64_t b = 0; b < r->nblocks; b++) {
        const int l = q->lijk[4 * b];
        if (l < 0 || l >= r->nlevels || (b > 0 && l < q->lijk[4 * (b - 1)])) return OHM_ERR_INVALID;
        q->lev_n[l]++;
    }
    for (int l = 1; l < r->nlevels; l++) q->lev_off[l] = q->lev_off[l - 1] + q->lev_n[l - 1];
    q->B.assign(r->B, r->B + (size_t)r->nblocks * B3C);
    q->eta.assign(r->eta, r->eta + (size_t)r->nblocks * B1C);
    q->dt = r->dt;
    q->nsteps = r->nsteps;
    q->out = r->B_out;
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stopping) return OHM_ERR_INVALID;
    const int64_t need = batch_bytes(S, q.get(), 1);  // also validates the structure
    if (need < 0 || need > S->d.hbm_budget_bytes) return OHM_ERR_INVALID;
    q->id = S->next_id++;
    q->res.t_submit = S->now();
    *id = q->id;
    S->queue.push_back(q.get());
    S->reqs[q->id] = std::move(q);
    S->cv_work.notify_all();
    return OHM_OK;
}

int ohm_server_wait(ohm_server *S, int64_t id, double timeout_s, ohm_request_result *res) {
    if (!S) return OHM_ERR_INVALID;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return OHM_ERR_INVALID;
    Req *r = it->second.get();
    auto ready = [&] { return r->done; };
    if (timeout_s < 0) S->cv_done.wait(lk, ready);
    else if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) return OHM_ERR_TIMEOUT;
    if (res) *res = r->res;
    S->reqs.erase(it);
    return OHM_OK;
}

double ohm_server_clock(const ohm_server *S) { return S ? S->now() : 0.0; }

int ohm_server_get_stats(ohm_server *S, ohm_server_stats *st) {
    if (!S || !st) return OHM_ERR_INVALID;
    std::lock_guard<std::mutex> lk(S->mu);
    *st = S->st;
    st->bytes_resident = S->resident;
    st->mean_active_slots = S->st.steps_run ? S->active_sum / (double)S->st.steps_run : 0.0;
    st->kernel_launches = S->launches_freed;
    for (auto &b : S->batches)
        if (b->h) st->kernel_launches += ohm_launch_count(b->h);
    return OHM_OK;
}

void ohm_server_destroy(ohm_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
        S->cv_work.notify_all();
    }
    for (auto &t : S->workers) t.join();
    for (auto &b : S->batches) free_batch(b.get());
    delete S;
}

}  // extern "C"
