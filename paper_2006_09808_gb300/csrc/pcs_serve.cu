// pcs_serve.cu -- serving loop: continuous batching of volume reconstructions.
//
// A volume request (S slices of H x W, its lambda) is opened with
// pcs_serve_open and its slices arrive over time (pcs_serve_push: an
// interventional scan streaming slices).  A scheduler thread owned by the
// server
//   * admits open requests in arrival order when a slot (a CUDA stream) is
//     free and the request's device footprint fits the HBM budget
//     (field + mask + chi + the four state arrays: 25 B per voxel);
//   * as soon as slices of an admitted request have arrived, copies them to
//     the device and launches the fused iteration kernel on them (slices are
//     independent, so solving them in chunks gives the same chi as solving the
//     volume at once); chunks of different requests run concurrently on
//     their slots' streams;
//   * copies chi back, and when every slice of a request is done, records its
//     latency (completion - open) and frees its budget.
// Step sizes are tau = sigma = 1/L(H, W) (Sec. II.A pseudocode step 1), L the
// full-mask operator norm, computed once per slice size; the kernel variant
// of each size is the one the batch autotuner picks.  The primal/dual state of
// an admitted request stays in device memory until the request completes.
#include <cuda_runtime.h>

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

#include "../../include/pcs.h"
#include "pd_launch.cuh"

namespace pcs {
void build_dipole_tables(int H, int W, int b0_axis, std::vector<float>& dtab, std::vector<float>& ddtab);
void build_twiddles(int n, std::vector<float2>& tw);
pcs_status set_last_error(pcs_status st, const char* msg);
// any-size slices (pd_generic.cu)
struct GenSolver;
bool gen_supported(int H, int W);
cudaError_t gen_create(GenSolver** out, int H, int W, int max_slices, int b0_axis, int tv);
void gen_destroy(GenSolver* gs);
cudaError_t gen_enqueue(GenSolver* gs, const float* field, const unsigned char* mask, const float* weight,
                        float* chi, float* chibar, float* p, float* qx, float* qy, int S, double lambda, double tau,
                        double sigma, int n_iter, cudaStream_t st, int resume, const int* active,
                        const float* inv_den_slice, float2* spec);
}  // namespace pcs

namespace {

using Clock = std::chrono::steady_clock;

double seconds_since(Clock::time_point t0) {
    return std::chrono::duration<double>(Clock::now() - t0).count();
}

const pcs::KernelEntry* registry_find(int H, int W, int C, int kernel, int threads) {
    const pcs::KernelEntry* (*fns[])(int*) = {pcs::entries_64,  pcs::entries_128, pcs::entries_192,
                                               pcs::entries_256, pcs::entries_384, pcs::entries_512};
    for (auto fn : fns) {
        int n = 0;
        const pcs::KernelEntry* e = fn(&n);
        for (int k = 0; k < n; ++k)
            if (e[k].H == H && e[k].W == W && (C <= 0 || e[k].C == C) &&
                (kernel <= 0 || e[k].resident == (kernel == 2 ? 1 : 0)) && (threads <= 0 || e[k].threads == threads))
                return &e[k];
    }
    return nullptr;
}

// Slice sizes the loop serves: a compiled variant, or the any-size kernels.
bool served_size(int H, int W) { return registry_find(H, W, 0, 0, 0) != nullptr || pcs::gen_supported(H, W); }

// Half-spectrum bytes per voxel of a size run by the any-size kernels (0 for compiled sizes).
size_t spec_bytes(int H, int W, size_t voxels) {
    if (registry_find(H, W, 0, 0, 0)) return 0;
    return voxels / (size_t)W * (size_t)(W / 2 + 1) * sizeof(float2);
}

// Per slice size: kernel variant, tables and step size, shared by all slots.
struct SizeInfo {
    int H = 0, W = 0;
    const pcs::KernelEntry* entry = nullptr;
    pcs::GenSolver* gen = nullptr;  // any-size kernels (tables only; each slot holds its spectrum)
    int max_clusters = 1;
    double L = 0.0;
    float* dtab = nullptr;
    float* ddtab = nullptr;
    float2* twid = nullptr;
    pcs_tuning tuning{};
};

struct Chunk {
    int s0, n;
    cudaEvent_t done;
};

struct Request {
    long long id = 0;
    int H = 0, W = 0, S = 0;
    double lambda = 0.0;
    float* chi_host = nullptr;
    Clock::time_point t_open;
    // slices pushed by the client, not yet launched: (first slice, count, host field, host mask)
    struct Arrival {
        int s0, n;
        const float* field;
        const unsigned char* mask;
    };
    std::deque<Arrival> arrived;
    int pushed = 0, launched = 0, completed = 0;
    int slot = -1;  // -1 while waiting for admission
    size_t bytes = 0;
    std::vector<Chunk> chunks;  // launched, not yet completed
};

struct Slot {
    cudaStream_t stream = nullptr;
    long long req = -1;  // request occupying the slot
    // device arena of the occupying request
    float* field = nullptr;
    unsigned char* mask = nullptr;
    float* chi = nullptr;
    float* state = nullptr;  // chibar, p, qx, qy
    float2* spec = nullptr;  // half spectrum, for sizes run by the any-size kernels
    size_t cap_voxels = 0, cap_spec = 0;
};

}  // namespace

struct pcs_server {
    pcs_server_config cfg{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::thread worker;
    bool stop = false;
    long long next_id = 1;
    std::map<long long, Request> reqs;
    std::deque<long long> admit_queue;  // open requests in arrival order, not yet admitted
    std::vector<Slot> slots;
    std::map<std::pair<int, int>, SizeInfo> sizes;
    size_t bytes_in_use = 0;
    // completions not yet polled: (id, latency s)
    std::deque<std::pair<long long, double>> done;
    // statistics
    Clock::time_point t_first_open;
    bool any_open = false;
    double t_last_done = 0.0;
    long long n_done = 0;
    double voxel_iters_done = 0.0;
    std::vector<double> latencies;
    int peak_inflight = 0;
    size_t peak_bytes = 0;
    pcs_status worker_error = PCS_OK;
    std::string worker_error_text;
};

namespace {

constexpr size_t kBytesPerVoxel = 4 + 1 + 4 + 16;  // field, mask, chi, 4 state arrays

pcs_status size_setup(pcs_server* sv, int H, int W, SizeInfo** out) {
    auto key = std::make_pair(H, W);
    auto it = sv->sizes.find(key);
    if (it != sv->sizes.end()) {
        *out = &it->second;
        return PCS_OK;
    }
    SizeInfo si;
    si.H = H;
    si.W = W;
    // autotune once on a synthetic volume (and get L) through the batch solver
    pcs_batch* b = nullptr;
    pcs_options o;
    pcs_options_default(&o);
    cudaStream_t ts = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking);
    if (e != cudaSuccess) return pcs::set_last_error(PCS_ECUDA, "serve: stream create");
    pcs_status st = pcs_batch_create(&b, &o, sv->cfg.autotune, ts);
    const int S = 16;
    float *f = nullptr, *chi = nullptr;
    unsigned char* m = nullptr;
    if (st == PCS_OK) {
        if (cudaMalloc(&f, (size_t)S * H * W * 4) != cudaSuccess || cudaMalloc(&chi, (size_t)S * H * W * 4) != cudaSuccess ||
            cudaMalloc(&m, (size_t)S * H * W) != cudaSuccess)
            st = pcs::set_last_error(PCS_ENOMEM, "serve: tuning buffers");
    }
    if (st == PCS_OK) {
        cudaMemsetAsync(f, 0, (size_t)S * H * W * 4, ts);
        cudaMemsetAsync(m, 1, (size_t)S * H * W, ts);
        pcs_volume v{H, W, S, 0, 1.0, f, m, chi};
        st = pcs_batch_solve(b, &v, 1, 4);
        if (st == PCS_OK && cudaStreamSynchronize(ts) != cudaSuccess) st = pcs::set_last_error(PCS_ECUDA, "serve: sync");
        if (st == PCS_OK) st = pcs_batch_tuning(b, H, W, &si.tuning);
    }
    if (b) pcs_batch_destroy(b);
    if (f) cudaFree(f);
    if (chi) cudaFree(chi);
    if (m) cudaFree(m);
    cudaStreamDestroy(ts);
    if (st != PCS_OK) return st;
    si.L = si.tuning.L;
    si.entry = registry_find(H, W, si.tuning.cluster_size, si.tuning.kernel, si.tuning.threads);
    if (!si.entry && pcs::gen_supported(H, W)) {
        if (!(si.L > 0.0) || pcs::gen_create(&si.gen, H, W, 1, sv->cfg.b0_axis, 0) != cudaSuccess)
            return pcs::set_last_error(PCS_ECUDA, "serve: any-size set-up");
        auto res = sv->sizes.emplace(key, si);
        *out = &res.first->second;
        return PCS_OK;
    }
    if (!si.entry || !(si.L > 0.0)) return pcs::set_last_error(PCS_ECUDA, "serve: size set-up");
    int aux = 0;
    if (si.entry->prepare(&si.max_clusters, &aux) != cudaSuccess) return pcs::set_last_error(PCS_ECUDA, "serve: prepare");
    std::vector<float> dtab, ddtab;
    std::vector<float2> tw;
    pcs::build_dipole_tables(H, W, sv->cfg.b0_axis, dtab, ddtab);
    pcs::build_twiddles(H > W ? H : W, tw);
    if (cudaMalloc(&si.dtab, dtab.size() * 4) != cudaSuccess || cudaMalloc(&si.ddtab, ddtab.size() * 4) != cudaSuccess ||
        cudaMalloc(&si.twid, tw.size() * sizeof(float2)) != cudaSuccess ||
        cudaMemcpy(si.dtab, dtab.data(), dtab.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(si.ddtab, ddtab.data(), ddtab.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(si.twid, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess)
        return pcs::set_last_error(PCS_ENOMEM, "serve: tables");
    auto res = sv->sizes.emplace(key, si);
    *out = &res.first->second;
    return PCS_OK;
}

void slot_release(Slot& sl) {
    void* p[] = {sl.field, sl.mask, sl.chi, sl.state, sl.spec};
    for (void* q : p)
        if (q) cudaFree(q);
    sl.field = nullptr;
    sl.mask = nullptr;
    sl.chi = nullptr;
    sl.state = nullptr;
    sl.spec = nullptr;
    sl.cap_voxels = 0;
    sl.cap_spec = 0;
}

// Admit waiting requests (arrival order) while a slot and budget are free.
void admit(pcs_server* sv) {
    while (!sv->admit_queue.empty()) {
        const long long id = sv->admit_queue.front();
        auto it = sv->reqs.find(id);
        if (it == sv->reqs.end()) {
            sv->admit_queue.pop_front();
            continue;
        }
        Request& r = it->second;
        int free_slot = -1;
        for (size_t k = 0; k < sv->slots.size(); ++k)
            if (sv->slots[k].req < 0) {
                free_slot = (int)k;
                break;
            }
        if (free_slot < 0) return;
        if (sv->bytes_in_use + r.bytes > sv->cfg.hbm_budget_bytes) return;  // wait for memory
        Slot& sl = sv->slots[free_slot];
        const size_t vox = (size_t)r.S * r.H * r.W;
        const size_t sb = spec_bytes(r.H, r.W, vox);
        if (sl.cap_voxels < vox || sl.cap_spec < sb) {
            slot_release(sl);
            if (cudaMalloc(&sl.field, vox * 4) != cudaSuccess || cudaMalloc(&sl.mask, vox) != cudaSuccess ||
                cudaMalloc(&sl.chi, vox * 4) != cudaSuccess || cudaMalloc(&sl.state, 4 * vox * 4) != cudaSuccess ||
                (sb > 0 && cudaMalloc(&sl.spec, sb) != cudaSuccess)) {
                slot_release(sl);
                return;  // device memory exhausted beyond the budget: retry later
            }
            sl.cap_voxels = vox;
            sl.cap_spec = sb;
        }
        sl.req = id;
        r.slot = free_slot;
        sv->bytes_in_use += r.bytes;
        sv->peak_bytes = std::max(sv->peak_bytes, sv->bytes_in_use);
        sv->admit_queue.pop_front();
        int inflight = 0;
        for (auto& s : sv->slots) inflight += s.req >= 0;
        sv->peak_inflight = std::max(sv->peak_inflight, inflight);
    }
}

// Launch every arrived slice range of admitted requests.
bool launch_arrived(pcs_server* sv) {
    bool any = false;
    for (auto& kv : sv->reqs) {
        Request& r = kv.second;
        if (r.slot < 0 || r.arrived.empty()) continue;
        Slot& sl = sv->slots[r.slot];
        SizeInfo* si = nullptr;
        if (size_setup(sv, r.H, r.W, &si) != PCS_OK) {
            sv->worker_error = PCS_ECUDA;
            sv->worker_error_text = "size set-up failed";
            continue;
        }
        const size_t slice = (size_t)r.H * r.W;
        const size_t vox = (size_t)r.S * slice;
        while (!r.arrived.empty()) {
            Request::Arrival a = r.arrived.front();
            r.arrived.pop_front();
            cudaError_t e1 =
                cudaMemcpyAsync(sl.field + a.s0 * slice, a.field, a.n * slice * 4, cudaMemcpyHostToDevice, sl.stream);
            cudaError_t e2 = cudaMemcpyAsync(sl.mask + a.s0 * slice, a.mask, a.n * slice, cudaMemcpyHostToDevice, sl.stream);
            cudaError_t e3 = cudaSuccess;
            if (si->gen) {
                // any-size kernels on this slot's stream and spectrum
                const double step = 1.0 / si->L;
                const size_t sp_slice = (size_t)r.H * (r.W / 2 + 1);
                e3 = pcs::gen_enqueue(si->gen, sl.field + a.s0 * slice, sl.mask + a.s0 * slice, nullptr,
                                      sl.chi + a.s0 * slice, sl.state + a.s0 * slice, sl.state + vox + a.s0 * slice,
                                      sl.state + 2 * vox + a.s0 * slice, sl.state + 3 * vox + a.s0 * slice, a.n,
                                      r.lambda, step, step, sv->cfg.n_iter, sl.stream, 0, nullptr, nullptr,
                                      sl.spec + a.s0 * sp_slice);
            }
            pcs::PDParams prm;
            std::memset(&prm, 0, sizeof(prm));
            prm.field = sl.field + a.s0 * slice;
            prm.mask = sl.mask + a.s0 * slice;
            prm.chi = sl.chi + a.s0 * slice;
            prm.chibar = sl.state + a.s0 * slice;
            prm.p = sl.state + vox + a.s0 * slice;
            prm.qx = sl.state + 2 * vox + a.s0 * slice;
            prm.qy = sl.state + 3 * vox + a.s0 * slice;
            prm.dtab = si->dtab;
            prm.ddtab = si->ddtab;
            prm.twid = si->twid;
            prm.S = a.n;
            prm.n_iter = sv->cfg.n_iter;
            prm.sigma = (float)(1.0 / si->L);
            prm.tau = (float)(1.0 / si->L);
            prm.inv_den = (float)(1.0 / (1.0 + (1.0 / si->L) / r.lambda));
            prm.inv_den_slice = nullptr;
            int ncl = std::min(si->max_clusters, a.n);
            if (!si->gen) e3 = si->entry->launch(prm, ncl < 1 ? 1 : ncl, sl.stream);
            cudaError_t e4 = cudaMemcpyAsync(r.chi_host + a.s0 * slice, sl.chi + a.s0 * slice, a.n * slice * 4,
                                             cudaMemcpyDeviceToHost, sl.stream);
            if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess || e4 != cudaSuccess) {
                sv->worker_error = PCS_ECUDA;
                sv->worker_error_text = "copy or launch failed in the serving loop";
            }
            Chunk c{a.s0, a.n, nullptr};
            cudaEventCreateWithFlags(&c.done, cudaEventDisableTiming);
            cudaEventRecord(c.done, sl.stream);
            r.chunks.push_back(c);
            r.launched += a.n;
            any = true;
        }
    }
    return any;
}

// Retire finished chunks and requests.
bool retire(pcs_server* sv) {
    bool any = false;
    std::vector<long long> finished;
    for (auto& kv : sv->reqs) {
        Request& r = kv.second;
        for (size_t k = 0; k < r.chunks.size();) {
            if (cudaEventQuery(r.chunks[k].done) == cudaSuccess) {
                r.completed += r.chunks[k].n;
                cudaEventDestroy(r.chunks[k].done);
                r.chunks.erase(r.chunks.begin() + k);
                any = true;
            } else {
                ++k;
            }
        }
        if (r.slot >= 0 && r.completed == r.S) finished.push_back(r.id);
    }
    for (long long id : finished) {
        Request& r = sv->reqs[id];
        const double lat = seconds_since(r.t_open);
        sv->slots[r.slot].req = -1;
        sv->bytes_in_use -= r.bytes;
        sv->done.emplace_back(id, lat);
        sv->latencies.push_back(lat);
        sv->n_done++;
        sv->voxel_iters_done += (double)r.S * r.H * r.W * sv->cfg.n_iter;
        sv->t_last_done = seconds_since(sv->t_first_open);
        sv->reqs.erase(id);
    }
    return any;
}

void worker_main(pcs_server* sv) {
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    while (!sv->stop) {
        admit(sv);
        const bool a = launch_arrived(sv);
        const bool b = retire(sv);
        if (!a && !b) {
            bool busy = false;
            for (auto& s : sv->slots) busy |= s.req >= 0;
            // short sleeps while work is on the GPU, else wait for a submission
            sv->cv.wait_for(lk, busy ? std::chrono::microseconds(200) : std::chrono::milliseconds(20));
        }
    }
}

}  // namespace

extern "C" {

pcs_status pcs_serve_start(pcs_server** out, const pcs_server_config* cfg) {
    if (!out || !cfg) return pcs::set_last_error(PCS_EINVAL, "pcs_serve_start: NULL argument");
    *out = nullptr;
    if (cfg->slots < 1 || cfg->n_iter < 0 || cfg->hbm_budget_bytes == 0)
        return pcs::set_last_error(PCS_EINVAL, "pcs_serve_start: slots >= 1, n_iter >= 0, budget > 0");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return pcs::set_last_error(PCS_ECUDA, "no CUDA device");
    pcs_server* sv = new pcs_server();
    sv->cfg = *cfg;
    cudaGetDevice(&sv->device);
    sv->slots.resize(cfg->slots);
    for (auto& s : sv->slots)
        if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess) {
            pcs_serve_stop(sv);
            return pcs::set_last_error(PCS_ECUDA, "pcs_serve_start: stream create");
        }
    sv->worker = std::thread(worker_main, sv);
    *out = sv;
    return PCS_OK;
}

pcs_status pcs_serve_prepare_size(pcs_server* sv, int H, int W, pcs_tuning* info) {
    if (!sv) return pcs::set_last_error(PCS_EINVAL, "server is NULL");
    if (!served_size(H, W)) return pcs::set_last_error(PCS_EUNSUPPORTED, "unsupported slice size");
    std::lock_guard<std::mutex> lk(sv->mu);
    SizeInfo* si = nullptr;
    pcs_status st = size_setup(sv, H, W, &si);
    if (st == PCS_OK && info) *info = si->tuning;
    return st;
}

pcs_status pcs_serve_open(pcs_server* sv, int H, int W, int S, double lambda, float* chi_host, long long* id) {
    if (!sv || !chi_host || !id) return pcs::set_last_error(PCS_EINVAL, "pcs_serve_open: NULL argument");
    if (S < 1 || !(lambda > 0.0)) return pcs::set_last_error(PCS_EINVAL, "pcs_serve_open: S >= 1 and lambda > 0");
    if (!served_size(H, W)) return pcs::set_last_error(PCS_EUNSUPPORTED, "pcs_serve_open: unsupported slice size");
    const size_t bytes = (size_t)S * H * W * kBytesPerVoxel + spec_bytes(H, W, (size_t)S * H * W);
    if (bytes > sv->cfg.hbm_budget_bytes) return pcs::set_last_error(PCS_ENOMEM, "pcs_serve_open: volume exceeds the budget");
    std::lock_guard<std::mutex> lk(sv->mu);
    Request r;
    r.id = sv->next_id++;
    r.H = H;
    r.W = W;
    r.S = S;
    r.lambda = lambda;
    r.chi_host = chi_host;
    r.t_open = Clock::now();
    r.bytes = bytes;
    if (!sv->any_open) {
        sv->any_open = true;
        sv->t_first_open = r.t_open;
    }
    sv->reqs.emplace(r.id, std::move(r));
    sv->admit_queue.push_back(*id = sv->next_id - 1);
    sv->cv.notify_one();
    return PCS_OK;
}

pcs_status pcs_serve_push(pcs_server* sv, long long id, int s0, int n, const float* field_host,
                          const unsigned char* mask_host) {
    if (!sv || !field_host || !mask_host) return pcs::set_last_error(PCS_EINVAL, "pcs_serve_push: NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(id);
    if (it == sv->reqs.end()) return pcs::set_last_error(PCS_EINVAL, "pcs_serve_push: unknown request");
    Request& r = it->second;
    if (n < 1 || s0 < 0 || s0 + n > r.S || s0 != r.pushed)
        return pcs::set_last_error(PCS_EINVAL, "pcs_serve_push: slices must arrive in order, within [0, S)");
    r.arrived.push_back({s0, n, field_host, mask_host});
    r.pushed += n;
    sv->cv.notify_one();
    return PCS_OK;
}

pcs_status pcs_serve_poll(pcs_server* sv, long long* ids, double* latency_s, int max, int* n_out) {
    if (!sv || !n_out || (max > 0 && (!ids || !latency_s))) return pcs::set_last_error(PCS_EINVAL, "pcs_serve_poll: NULL");
    std::lock_guard<std::mutex> lk(sv->mu);
    int n = 0;
    while (n < max && !sv->done.empty()) {
        ids[n] = sv->done.front().first;
        latency_s[n] = sv->done.front().second;
        sv->done.pop_front();
        ++n;
    }
    *n_out = n;
    return sv->worker_error;
}

pcs_status pcs_serve_stats(pcs_server* sv, pcs_serve_summary* out) {
    if (!sv || !out) return pcs::set_last_error(PCS_EINVAL, "pcs_serve_stats: NULL");
    std::lock_guard<std::mutex> lk(sv->mu);
    std::memset(out, 0, sizeof(*out));
    out->completed = sv->n_done;
    out->pending = (long long)sv->reqs.size();
    out->voxel_iters = sv->voxel_iters_done;
    out->span_s = sv->t_last_done;
    out->peak_inflight = sv->peak_inflight;
    out->peak_bytes = (double)sv->peak_bytes;
    std::vector<double> l = sv->latencies;
    if (!l.empty()) {
        std::sort(l.begin(), l.end());
        auto q = [&](double f) { return l[std::min(l.size() - 1, (size_t)(f * (l.size() - 1) + 0.5))]; };
        out->p50_s = q(0.50);
        out->p99_s = q(0.99);
        out->max_s = l.back();
    }
    return PCS_OK;
}

void pcs_serve_stop(pcs_server* sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        sv->cv.notify_all();
    }
    if (sv->worker.joinable()) sv->worker.join();
    for (auto& s : sv->slots) {
        if (s.stream) cudaStreamSynchronize(s.stream);
        slot_release(s);
        if (s.stream) cudaStreamDestroy(s.stream);
    }
    for (auto& kv : sv->reqs)
        for (auto& c : kv.second.chunks) cudaEventDestroy(c.done);
    for (auto& kv : sv->sizes) {
        cudaFree(kv.second.dtab);
        cudaFree(kv.second.ddtab);
        cudaFree(kv.second.twid);
        pcs::gen_destroy(kv.second.gen);
    }
    delete sv;
}

}  // extern "C"
