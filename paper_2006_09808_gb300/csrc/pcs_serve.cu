// pcs_serve.cu -- serving loop: continuous batching of volume reconstructions.
//
// A volume request (S slices of H x W, its lambda) is opened with
// pcs_serve_open and its slices arrive over time (pcs_serve_push: an
// interventional scan streaming slices).  The server allocates one device
// arena of the HBM budget when it starts; a scheduler thread owned by the
// server
//   * admits open requests in arrival order when a slot (a CUDA stream) is
//     free and the request's device footprint (field + mask + chi + the four
//     state arrays, 25 B per voxel, plus the half spectrum for sizes run by
//     the any-size kernels) fits in a free range of the arena -- the budget is
//     exactly the memory the requests hold, and the scheduler thread never
//     allocates or frees device memory;
//   * as soon as slices of an admitted request have arrived, copies them to
//     the device and launches the fused iteration kernel on them (slices are
//     independent, so solving them in chunks gives the same chi as solving the
//     volume at once); chunks of different requests run concurrently on
//     their slots' streams;
//   * copies chi back, and when every slice of a request is done, records its
//     latency (completion - open) and returns its range to the arena.
// A request whose copy or launch fails is finished alone with that status
// (its remaining slices are not launched); the other requests go on.  A
// sticky CUDA error (a device fault) ends the server: pcs_serve_poll
// reports it.
// Step sizes are tau = sigma = 1/L(H, W) (Sec. II.A pseudocode step 1), L the
// full-mask operator norm, computed once per slice size; the kernel variant
// of each size is the one the batch autotuner picks.  The primal/dual state of
// an admitted request stays in device memory until the request completes.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <iterator>
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

const pcs::KernelEntry* registry_find(int H, int W, int C, int kernel, int threads, int tile = 0) {
    const pcs::KernelEntry* (*fns[])(int*) = {pcs::entries_64,  pcs::entries_128, pcs::entries_192,
                                               pcs::entries_256, pcs::entries_384, pcs::entries_512};
    for (auto fn : fns) {
        int n = 0;
        const pcs::KernelEntry* e = fn(&n);
        for (int k = 0; k < n; ++k)
            if (e[k].H == H && e[k].W == W && (C <= 0 || e[k].C == C) &&
                (kernel <= 0 || e[k].resident == (kernel == 2 ? 1 : 0)) && (threads <= 0 || e[k].threads == threads) &&
                (tile <= 0 || e[k].tile == tile))
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
    cudaEvent_t done;  // recorded after the chunk's copies and launch
    bool ok;           // false: a copy or launch of the chunk failed (its slices are dropped)
};

// First-fit allocator of byte ranges inside the server's device arena (host bookkeeping only).
class Arena {
  public:
    static constexpr size_t kAlign = 256;
    void reset(size_t cap) {
        free_.clear();
        if (cap) free_[0] = cap;
        used_ = 0;
    }
    // offset of a free range of `bytes` (a multiple of kAlign), or SIZE_MAX
    size_t alloc(size_t bytes) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            const size_t off = it->first, len = it->second;
            free_.erase(it);
            if (len > bytes) free_[off + bytes] = len - bytes;
            used_ += bytes;
            return off;
        }
        return SIZE_MAX;
    }
    void release(size_t off, size_t bytes) {
        used_ -= bytes;
        auto nx = free_.lower_bound(off);
        if (nx != free_.end() && off + bytes == nx->first) {  // merge with the next range
            bytes += nx->second;
            nx = free_.erase(nx);
        }
        if (nx != free_.begin()) {  // merge with the previous range
            auto pv = std::prev(nx);
            if (pv->first + pv->second == off) {
                pv->second += bytes;
                return;
            }
        }
        free_[off] = bytes;
    }
    size_t used() const { return used_; }

  private:
    std::map<size_t, size_t> free_;  // offset -> length
    size_t used_ = 0;
};

size_t align_up(size_t n) { return (n + Arena::kAlign - 1) / Arena::kAlign * Arena::kAlign; }

// Device bytes a request holds: field, mask, chi, chibar/p/qx/qy and (any-size kernels) the half
// spectrum, each range 256-byte aligned.
size_t request_bytes(int H, int W, int S) {
    const size_t vox = (size_t)S * H * W;
    return align_up(vox * 4) + align_up(vox) + align_up(vox * 4) + align_up(4 * vox * 4) +
           align_up(spec_bytes(H, W, vox));
}

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
    int pushed = 0, launched = 0, completed = 0, dropped = 0;
    int slot = -1;  // -1 while waiting for admission
    size_t bytes = 0;
    size_t arena_off = SIZE_MAX;  // its range of the arena once admitted
    // device buffers inside that range
    float* field = nullptr;
    unsigned char* mask = nullptr;
    float* chi = nullptr;
    float* state = nullptr;  // chibar, p, qx, qy
    float2* spec = nullptr;  // half spectrum, for sizes run by the any-size kernels
    pcs_status st = PCS_OK;  // a failed copy or launch finishes the request with this status
    bool fail_next = false;  // host-side fault injection (tests): the next launch reports failure
    std::vector<Chunk> chunks;  // launched, not yet completed
};

struct Slot {
    cudaStream_t stream = nullptr;
    long long req = -1;  // request occupying the slot
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
    char* arena_base = nullptr;  // one device allocation of hbm_budget_bytes, made at start
    Arena arena;
    std::vector<cudaEvent_t> events;  // pool of chunk-completion events (created at start, reused)
    // completions not yet polled: (id, latency s, status)
    struct Done {
        long long id;
        double latency;
        pcs_status st;
    };
    std::deque<Done> done;
    // statistics
    Clock::time_point t_first_open;
    bool any_open = false;
    double t_last_done = 0.0;
    long long n_done = 0;
    double voxel_iters_done = 0.0;
    std::vector<double> latencies;
    int peak_inflight = 0;
    size_t peak_bytes = 0;
    long long n_failed = 0;
    pcs_status worker_error = PCS_OK;  // server-level (sticky) CUDA error
    std::string worker_error_text;
};

namespace {

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
    si.entry = registry_find(H, W, si.tuning.cluster_size, si.tuning.kernel, si.tuning.threads, si.tuning.tile);
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

// Admit waiting requests (arrival order) while a slot and a large enough arena range are free.
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
        const size_t off = sv->arena.alloc(r.bytes);
        if (off == SIZE_MAX) return;  // wait for memory (arrival order: no overtaking)
        r.arena_off = off;
        const size_t vox = (size_t)r.S * r.H * r.W;
        char* p = sv->arena_base + off;
        r.field = reinterpret_cast<float*>(p);
        p += align_up(vox * 4);
        r.mask = reinterpret_cast<unsigned char*>(p);
        p += align_up(vox);
        r.chi = reinterpret_cast<float*>(p);
        p += align_up(vox * 4);
        r.state = reinterpret_cast<float*>(p);
        p += align_up(4 * vox * 4);
        r.spec = spec_bytes(r.H, r.W, vox) ? reinterpret_cast<float2*>(p) : nullptr;
        sv->slots[free_slot].req = id;
        r.slot = free_slot;
        sv->peak_bytes = std::max(sv->peak_bytes, sv->arena.used());
        sv->admit_queue.pop_front();
        int inflight = 0;
        for (auto& s : sv->slots) inflight += s.req >= 0;
        sv->peak_inflight = std::max(sv->peak_inflight, inflight);
    }
}

// Launch every arrived slice range of admitted requests.  A request whose copy or launch fails
// gets that status; its later slices are dropped.
bool launch_arrived(pcs_server* sv) {
    bool any = false;
    for (auto& kv : sv->reqs) {
        Request& r = kv.second;
        if (r.slot < 0 || r.arrived.empty()) continue;
        Slot& sl = sv->slots[r.slot];
        auto sit = sv->sizes.find(std::make_pair(r.H, r.W));
        SizeInfo* si = sit == sv->sizes.end() ? nullptr : &sit->second;  // set up when the request opened
        const size_t slice = (size_t)r.H * r.W;
        const size_t vox = (size_t)r.S * slice;
        while (!r.arrived.empty()) {
            Request::Arrival a = r.arrived.front();
            r.arrived.pop_front();
            any = true;
            if (r.st != PCS_OK || !si) {  // a failed request launches nothing more
                if (r.st == PCS_OK) r.st = PCS_EINVAL;
                r.dropped += a.n;
                continue;
            }
            cudaError_t e1 =
                cudaMemcpyAsync(r.field + a.s0 * slice, a.field, a.n * slice * 4, cudaMemcpyHostToDevice, sl.stream);
            cudaError_t e2 = cudaMemcpyAsync(r.mask + a.s0 * slice, a.mask, a.n * slice, cudaMemcpyHostToDevice, sl.stream);
            cudaError_t e3 = cudaSuccess;
            if (si->gen) {
                // any-size kernels on this slot's stream and the request's spectrum
                const double step = 1.0 / si->L;
                const size_t sp_slice = (size_t)r.H * (r.W / 2 + 1);
                e3 = pcs::gen_enqueue(si->gen, r.field + a.s0 * slice, r.mask + a.s0 * slice, nullptr,
                                      r.chi + a.s0 * slice, r.state + a.s0 * slice, r.state + vox + a.s0 * slice,
                                      r.state + 2 * vox + a.s0 * slice, r.state + 3 * vox + a.s0 * slice, a.n,
                                      r.lambda, step, step, sv->cfg.n_iter, sl.stream, 0, nullptr, nullptr,
                                      r.spec + a.s0 * sp_slice);
            } else {
                pcs::PDParams prm;
                std::memset(&prm, 0, sizeof(prm));
                prm.field = r.field + a.s0 * slice;
                prm.mask = r.mask + a.s0 * slice;
                prm.chi = r.chi + a.s0 * slice;
                prm.chibar = r.state + a.s0 * slice;
                prm.p = r.state + vox + a.s0 * slice;
                prm.qx = r.state + 2 * vox + a.s0 * slice;
                prm.qy = r.state + 3 * vox + a.s0 * slice;
                prm.dtab = si->dtab;
                prm.ddtab = si->ddtab;
                prm.twid = si->twid;
                prm.S = a.n;
                prm.n_iter = sv->cfg.n_iter;
                prm.sigma = (float)(1.0 / si->L);
                prm.tau = (float)(1.0 / si->L);
                prm.inv_den = (float)(1.0 / (1.0 + (1.0 / si->L) / r.lambda));
                prm.inv_den_slice = nullptr;
                const int ncl = std::min(si->max_clusters, a.n);
                e3 = si->entry->launch(prm, ncl < 1 ? 1 : ncl, sl.stream);
            }
            if (r.fail_next) {  // injected on the host: this launch reports an error code
                r.fail_next = false;
                e3 = cudaErrorLaunchOutOfResources;
            }
            cudaError_t e4 = cudaMemcpyAsync(r.chi_host + a.s0 * slice, r.chi + a.s0 * slice, a.n * slice * 4,
                                             cudaMemcpyDeviceToHost, sl.stream);
            const bool ok = e1 == cudaSuccess && e2 == cudaSuccess && e3 == cudaSuccess && e4 == cudaSuccess;
            if (!ok) {
                // this request fails alone; a sticky error (the context is lost) stops the server
                r.st = PCS_ECUDA;
                (void)cudaGetLastError();  // clears a non-sticky error
                if (cudaGetLastError() != cudaSuccess) {
                    sv->worker_error = PCS_ECUDA;
                    sv->worker_error_text = "sticky CUDA error in the serving loop";
                }
            }
            // whatever was enqueued must finish before the request's arena range is reused
            Chunk c{a.s0, a.n, nullptr, ok};
            if (sv->events.empty()) {  // pool exhausted (many chunks in flight): one more event
                cudaEvent_t ev = nullptr;
                if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess) sv->events.push_back(ev);
            }
            if (!sv->events.empty()) {
                c.done = sv->events.back();
                sv->events.pop_back();
            }
            if (!c.done || cudaEventRecord(c.done, sl.stream) != cudaSuccess) {
                if (c.done) sv->events.push_back(c.done);
                c.done = nullptr;
                cudaStreamSynchronize(sl.stream);
                c.ok = false;
                r.st = PCS_ECUDA;
            }
            r.chunks.push_back(c);
            r.launched += a.n;
        }
    }
    return any;
}

// Retire finished chunks and requests (a failed request once none of its chunks is in flight
// and every slice was pushed or it can no longer complete).
bool retire(pcs_server* sv) {
    bool any = false;
    std::vector<long long> finished;
    for (auto& kv : sv->reqs) {
        Request& r = kv.second;
        for (size_t k = 0; k < r.chunks.size();) {
            const cudaError_t q = r.chunks[k].done ? cudaEventQuery(r.chunks[k].done) : cudaSuccess;
            if (q != cudaErrorNotReady) {
                if (q == cudaSuccess && r.chunks[k].ok) {
                    r.completed += r.chunks[k].n;
                } else {
                    r.st = PCS_ECUDA;
                    r.dropped += r.chunks[k].n;
                }
                if (r.chunks[k].done) sv->events.push_back(r.chunks[k].done);  // back to the pool
                r.chunks.erase(r.chunks.begin() + k);
                any = true;
            } else {
                ++k;
            }
        }
        if (r.slot < 0 || !r.chunks.empty()) continue;
        if (r.completed == r.S || (r.st != PCS_OK && r.arrived.empty())) finished.push_back(r.id);
    }
    for (long long id : finished) {
        Request& r = sv->reqs[id];
        const double lat = seconds_since(r.t_open);
        sv->slots[r.slot].req = -1;
        sv->arena.release(r.arena_off, r.bytes);
        sv->done.push_back({id, lat, r.st});
        if (r.st == PCS_OK) {
            sv->latencies.push_back(lat);
            sv->n_done++;
            sv->voxel_iters_done += (double)r.S * r.H * r.W * sv->cfg.n_iter;
            sv->t_last_done = seconds_since(sv->t_first_open);
        } else {
            sv->n_failed++;
        }
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
    // the whole budget, once: requests are placed in it and the scheduler never allocates
    const size_t cap = cfg->hbm_budget_bytes / Arena::kAlign * Arena::kAlign;
    if (cap == 0 || cudaMalloc(&sv->arena_base, cap) != cudaSuccess) {
        sv->arena_base = nullptr;
        pcs_serve_stop(sv);
        return pcs::set_last_error(PCS_ENOMEM, "pcs_serve_start: cannot allocate the budget's device arena");
    }
    sv->arena.reset(cap);
    for (int k = 0; k < 16 * cfg->slots; ++k) {
        cudaEvent_t ev = nullptr;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            pcs_serve_stop(sv);
            return pcs::set_last_error(PCS_ECUDA, "pcs_serve_start: event create");
        }
        sv->events.push_back(ev);
    }
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
    const size_t bytes = request_bytes(H, W, S);
    if (bytes > sv->cfg.hbm_budget_bytes / Arena::kAlign * Arena::kAlign)
        return pcs::set_last_error(PCS_ENOMEM, "pcs_serve_open: volume exceeds the budget");
    std::lock_guard<std::mutex> lk(sv->mu);
    // a new slice size is set up here, on the caller's thread (autotuning, tables, step size)
    SizeInfo* si = nullptr;
    pcs_status st = size_setup(sv, H, W, &si);
    if (st != PCS_OK) return st;
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

pcs_status pcs_serve_poll(pcs_server* sv, long long* ids, double* latency_s, pcs_status* status, int max,
                          int* n_out) {
    if (!sv || !n_out || (max > 0 && (!ids || !latency_s))) return pcs::set_last_error(PCS_EINVAL, "pcs_serve_poll: NULL");
    std::lock_guard<std::mutex> lk(sv->mu);
    int n = 0;
    while (n < max && !sv->done.empty()) {
        ids[n] = sv->done.front().id;
        latency_s[n] = sv->done.front().latency;
        if (status) status[n] = sv->done.front().st;
        sv->done.pop_front();
        ++n;
    }
    *n_out = n;
    if (sv->worker_error != PCS_OK) return pcs::set_last_error(sv->worker_error, sv->worker_error_text.c_str());
    return PCS_OK;
}

pcs_status pcs_serve_arena_plan(size_t capacity, const long long* ops, int n_ops, long long* offsets,
                                size_t* used_after) {
    if (!ops || !offsets || n_ops < 0) return pcs::set_last_error(PCS_EINVAL, "pcs_serve_arena_plan: bad argument");
    Arena a;
    const size_t cap = capacity / Arena::kAlign * Arena::kAlign;
    a.reset(cap);
    std::vector<std::pair<size_t, size_t>> held(n_ops, {SIZE_MAX, 0});  // by op index: (offset, bytes)
    for (int k = 0; k < n_ops; ++k) {
        offsets[k] = -1;
        if (ops[k] > 0) {  // allocate ops[k] bytes (rounded up to the alignment)
            const size_t b = align_up((size_t)ops[k]);
            const size_t off = a.alloc(b);
            if (off != SIZE_MAX) {
                held[k] = {off, b};
                offsets[k] = (long long)off;
            }
        } else if (ops[k] < 0) {  // release the range allocated by op -ops[k] - 1
            const long long j = -ops[k] - 1;
            if (j >= k || ops[j] <= 0)
                return pcs::set_last_error(PCS_EINVAL, "pcs_serve_arena_plan: release of an op that allocated nothing");
            if (held[j].first != SIZE_MAX) {  // a refused (or already released) allocation: nothing to do
                a.release(held[j].first, held[j].second);
                held[j] = {SIZE_MAX, 0};
            }
        }
        if (used_after) used_after[k] = a.used();
    }
    return PCS_OK;
}

pcs_status pcs_serve_request_bytes(int H, int W, int S, size_t* bytes) {
    if (!bytes || S < 1) return pcs::set_last_error(PCS_EINVAL, "pcs_serve_request_bytes: bad argument");
    if (!served_size(H, W)) return pcs::set_last_error(PCS_EUNSUPPORTED, "unsupported slice size");
    *bytes = request_bytes(H, W, S);
    return PCS_OK;
}

pcs_status pcs_serve_fail_next_launch(pcs_server* sv, long long id) {
    if (!sv) return pcs::set_last_error(PCS_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(id);
    if (it == sv->reqs.end()) return pcs::set_last_error(PCS_EINVAL, "pcs_serve_fail_next_launch: unknown request");
    it->second.fail_next = true;
    return PCS_OK;
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
    out->failed = sv->n_failed;
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
        if (s.stream) cudaStreamDestroy(s.stream);
    }
    for (auto& kv : sv->reqs)
        for (auto& c : kv.second.chunks)
            if (c.done) cudaEventDestroy(c.done);
    for (cudaEvent_t ev : sv->events) cudaEventDestroy(ev);
    if (sv->arena_base) cudaFree(sv->arena_base);
    for (auto& kv : sv->sizes) {
        cudaFree(kv.second.dtab);
        cudaFree(kv.second.ddtab);
        cudaFree(kv.second.twid);
        pcs::gen_destroy(kv.second.gen);
    }
    delete sv;
}

}  // extern "C"
