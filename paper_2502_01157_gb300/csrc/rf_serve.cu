// rf_serve.cu -- continuous-batching render server over a resident foam.
//
// The renderer of the paper (Sec. 3.4, "a (very) low overhead renderer")
// serves one frame at a time.  Here requests (a camera each, mixed
// resolutions) arrive asynchronously:
//   - admission by memory: each request reserves 20 B per ray (rgb, T,
//     depth) in a device pool sized by the caller, and a request slot;
//     otherwise rf_serve_submit returns RF_ERR_BUSY at once;
//   - a scheduler thread takes the admitted requests waiting to run and
//     launches them together (up to max_batch cameras of any sizes in one
//     multi-camera launch) on whichever of n_streams streams is free, so
//     requests that arrive while others are on the GPU start as soon as a
//     stream frees up and their work overlaps on the device;
//   - each launch is followed by the copy of the images to pinned host
//     memory and a host callback that stamps the completion time;
//   - rf_serve_poll hands the image over and releases the memory.
// The forward kernel computes every ray independently of the others, so an
// image is bit-identical whether it was rendered alone or in a batch.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "rf_host.h"

namespace rf {
rf_status launch_fwd_batch(const rf_scene *s, const rf_camera *cams, const int64_t *ray_offsets, int n,
                           float eps, int32_t max_steps, float *rgb, float *trans, float *depth,
                           unsigned long long *keys, cudaStream_t st);
}

using namespace rf;

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Req {
    rf_camera cam;
    int64_t off = 0, rays = 0;
    double t_submit = 0, t_done = 0;
    bool launched = false, done = false;
};

struct Batch;

}  // namespace

struct rf_server {
    rf_scene *scene = nullptr;
    rf_serve_config cfg{};
    float eps = 1e-4f;
    int32_t max_steps = kDefaultMaxSteps;
    int64_t cap = 0;  // pool capacity in rays
    float *d_rgb = nullptr, *d_trans = nullptr, *d_depth = nullptr;
    float *h_rgb = nullptr;  // pinned
    unsigned long long *d_keys = nullptr;  // [n_streams][kMaxCamsPerLaunch]
    std::vector<cudaStream_t> streams;
    std::vector<int> free_streams;
    std::map<int64_t, int64_t> free_ranges;  // offset -> length (rays)
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, Req> reqs;
    uint64_t next_id = 1;
    int inflight = 0;  // admitted, not yet released
    std::mutex mu;
    std::condition_variable cv;
    std::thread th;
    bool stop = false;
    rf_status thread_error = RF_OK;
    // statistics
    std::vector<double> lat_ms;
    int64_t rays_done = 0, rejected = 0, batches = 0, batch_reqs = 0, busy_streams_max = 0;
    double t_first = -1, t_last = 0;
};

namespace {

struct Batch {
    rf_server *srv;
    int stream;
    std::vector<uint64_t> ids;
};

bool pool_alloc(rf_server *s, int64_t n, int64_t *off) {
    for (auto it = s->free_ranges.begin(); it != s->free_ranges.end(); ++it) {
        if (it->second >= n) {
            *off = it->first;
            const int64_t rest = it->second - n, start = it->first + n;
            s->free_ranges.erase(it);
            if (rest > 0) s->free_ranges[start] = rest;
            return true;
        }
    }
    return false;
}

void pool_free(rf_server *s, int64_t off, int64_t n) {
    auto it = s->free_ranges.emplace(off, n).first;
    auto next = std::next(it);
    if (next != s->free_ranges.end() && it->first + it->second == next->first) {
        it->second += next->second;
        s->free_ranges.erase(next);
    }
    if (it != s->free_ranges.begin()) {
        auto prev = std::prev(it);
        if (prev->first + prev->second == it->first) {
            prev->second += it->second;
            s->free_ranges.erase(it);
        }
    }
}

void CUDART_CB batch_done(void *user) {
    Batch *b = static_cast<Batch *>(user);
    rf_server *s = b->srv;
    const double t = now_ms();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (uint64_t id : b->ids) {
            auto it = s->reqs.find(id);
            if (it == s->reqs.end()) continue;
            it->second.done = true;
            it->second.t_done = t;
            s->lat_ms.push_back(t - it->second.t_submit);
            s->rays_done += it->second.rays;
        }
        s->t_last = t;
        s->free_streams.push_back(b->stream);
    }
    s->cv.notify_all();
    delete b;
}

void scheduler(rf_server *s) {
    cudaSetDevice(s->scene->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        s->cv.wait(lk, [&] { return s->stop || (!s->pending.empty() && !s->free_streams.empty()); });
        if (s->stop) break;
        const int sid = s->free_streams.back();
        s->free_streams.pop_back();
        const int busy = (int)s->streams.size() - (int)s->free_streams.size();
        if (busy > s->busy_streams_max) s->busy_streams_max = busy;
        Batch *b = new Batch{s, sid, {}};
        std::vector<rf_camera> cams;
        std::vector<int64_t> offs;
        while (!s->pending.empty() && (int)b->ids.size() < s->cfg.max_batch) {
            const uint64_t id = s->pending.front();
            s->pending.pop_front();
            Req &r = s->reqs[id];
            r.launched = true;
            b->ids.push_back(id);
            cams.push_back(r.cam);
            offs.push_back(r.off);
        }
        s->batches += 1;
        s->batch_reqs += (int64_t)b->ids.size();
        lk.unlock();
        // launch outside the lock: nn(o) + forward for the whole batch, then
        // the images to pinned memory, then the completion callback
        cudaStream_t st = s->streams[sid];
        rf_status rc = launch_fwd_batch(s->scene, cams.data(), offs.data(), (int)cams.size(), s->eps,
                                        s->max_steps, s->d_rgb, s->d_trans, s->d_depth,
                                        s->d_keys + (size_t)sid * kMaxCamsPerLaunch, st);
        for (size_t k = 0; rc == RF_OK && k < cams.size(); ++k) {
            const int64_t n = (int64_t)cams[k].width * cams[k].height;
            if (cudaMemcpyAsync(s->h_rgb + 3 * offs[k], s->d_rgb + 3 * offs[k], sizeof(float) * 3 * n,
                                cudaMemcpyDeviceToHost, st) != cudaSuccess)
                rc = RF_ERR_CUDA;
        }
        if (rc == RF_OK && cudaLaunchHostFunc(st, batch_done, b) != cudaSuccess) rc = RF_ERR_CUDA;
        lk.lock();
        if (rc != RF_OK) {
            s->thread_error = rc;
            s->free_streams.push_back(sid);
            delete b;
            s->stop = true;
            s->cv.notify_all();
            break;
        }
    }
}

}  // namespace

RF_API rf_status rf_serve_create(rf_scene *scene, const rf_serve_config *cfg, rf_server **out) {
    if (!scene || !cfg || !out) return fail(RF_ERR_INVALID_ARG, "scene, cfg and out must not be NULL");
    *out = nullptr;
    if (cfg->max_inflight < 1 || cfg->n_streams < 1 || cfg->n_streams > 64 || cfg->max_batch < 1 ||
        cfg->max_batch > kMaxCamsPerLaunch)
        return fail(RF_ERR_INVALID_ARG, "need max_inflight >= 1, n_streams in [1,64], max_batch in [1,%d]",
                    kMaxCamsPerLaunch);
    float eps;
    int32_t max_steps;
    rf_render_opts o{};
    o.eps = cfg->eps;
    o.max_steps = cfg->max_steps;
    rf_status rc = check_opts(&o, &eps, &max_steps, nullptr);
    if (rc != RF_OK) return rc;
    rf_server *s = new rf_server();
    s->scene = scene;
    s->cfg = *cfg;
    s->eps = eps;
    s->max_steps = max_steps;
    s->cap = (int64_t)(cfg->mem_budget_bytes / 20);
    auto bail = [&](rf_status r) {
        cudaFree(s->d_rgb);
        cudaFree(s->d_trans);
        cudaFree(s->d_depth);
        cudaFree(s->d_keys);
        if (s->h_rgb) cudaFreeHost(s->h_rgb);
        for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
        delete s;
        return r;
    };
    cudaError_t ce;
    const int64_t cap = s->cap > 0 ? s->cap : 1;
    if ((ce = cudaMalloc(&s->d_rgb, sizeof(float) * 3 * cap)) != cudaSuccess ||
        (ce = cudaMalloc(&s->d_trans, sizeof(float) * cap)) != cudaSuccess ||
        (ce = cudaMalloc(&s->d_depth, sizeof(float) * cap)) != cudaSuccess ||
        (ce = cudaMalloc(&s->d_keys, sizeof(unsigned long long) * kMaxCamsPerLaunch * cfg->n_streams)) != cudaSuccess ||
        (ce = cudaMallocHost(&s->h_rgb, sizeof(float) * 3 * cap)) != cudaSuccess)
        return bail(cuda_fail(ce, "serve pool"));
    for (int k = 0; k < cfg->n_streams; ++k) {
        cudaStream_t st;
        if ((ce = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess)
            return bail(cuda_fail(ce, "serve stream"));
        s->streams.push_back(st);
        s->free_streams.push_back(k);
    }
    if (s->cap > 0) s->free_ranges[0] = s->cap;
    s->th = std::thread(scheduler, s);
    *out = s;
    return RF_OK;
}

RF_API rf_status rf_serve_submit(rf_server *s, const rf_camera *cam, uint64_t *req_id) {
    if (!s || !cam || !req_id) return fail(RF_ERR_INVALID_ARG, "server, cam and req_id must not be NULL");
    rf_status rc = check_camera(*cam, 0);
    if (rc != RF_OK) return rc;
    const int64_t n = (int64_t)cam->width * cam->height;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->thread_error != RF_OK) return fail(s->thread_error, "server scheduler stopped after a CUDA error");
    if (n > s->cap) {
        s->rejected += 1;
        return fail(RF_ERR_INVALID_ARG, "request of %lld rays exceeds the memory budget (%lld rays)",
                    (long long)n, (long long)s->cap);
    }
    int64_t off = 0;
    if (s->inflight >= s->cfg.max_inflight || !pool_alloc(s, n, &off)) {
        s->rejected += 1;
        return fail(RF_ERR_BUSY, "not admitted: %d requests in flight, memory for %lld rays not free",
                    s->inflight, (long long)n);
    }
    const uint64_t id = s->next_id++;
    Req &r = s->reqs[id];
    r.cam = *cam;
    r.off = off;
    r.rays = n;
    r.t_submit = now_ms();
    if (s->t_first < 0) s->t_first = r.t_submit;
    s->inflight += 1;
    s->pending.push_back(id);
    *req_id = id;
    s->cv.notify_all();
    return RF_OK;
}

static rf_status take_result(rf_server *s, std::unordered_map<uint64_t, Req>::iterator it, float *host_rgb,
                             double *latency_ms) {
    Req &r = it->second;
    if (host_rgb) memcpy(host_rgb, s->h_rgb + 3 * r.off, sizeof(float) * 3 * r.rays);
    if (latency_ms) *latency_ms = r.t_done - r.t_submit;
    pool_free(s, r.off, r.rays);
    s->inflight -= 1;
    s->reqs.erase(it);
    return RF_OK;
}

RF_API rf_status rf_serve_poll(rf_server *s, uint64_t req_id, float *host_rgb, int32_t *done,
                               double *latency_ms) {
    if (!s || !done) return fail(RF_ERR_INVALID_ARG, "server and done must not be NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end()) return fail(RF_ERR_NOT_FOUND, "unknown request %llu", (unsigned long long)req_id);
    *done = it->second.done ? 1 : 0;
    if (!it->second.done) return RF_OK;
    return take_result(s, it, host_rgb, latency_ms);
}

RF_API rf_status rf_serve_wait(rf_server *s, uint64_t req_id, int32_t timeout_ms, float *host_rgb,
                               double *latency_ms) {
    if (!s) return fail(RF_ERR_INVALID_ARG, "server must not be NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    auto ready = [&] {
        auto it = s->reqs.find(req_id);
        return it == s->reqs.end() || it->second.done || s->thread_error != RF_OK;
    };
    if (!s->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms), ready))
        return fail(RF_ERR_TIMEOUT, "request %llu not done after %d ms", (unsigned long long)req_id, timeout_ms);
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end()) return fail(RF_ERR_NOT_FOUND, "unknown request %llu", (unsigned long long)req_id);
    if (!it->second.done) return fail(s->thread_error, "server scheduler stopped after a CUDA error");
    return take_result(s, it, host_rgb, latency_ms);
}

RF_API rf_status rf_serve_stats(rf_server *s, rf_serve_metrics *out) {
    if (!s || !out) return fail(RF_ERR_INVALID_ARG, "server and out must not be NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    memset(out, 0, sizeof *out);
    std::vector<double> v = s->lat_ms;
    std::sort(v.begin(), v.end());
    auto pct = [&](double q) {
        if (v.empty()) return 0.0;
        const size_t k = (size_t)std::min<double>((double)v.size() - 1, std::ceil(q * v.size()) - 1);
        return v[k];
    };
    out->completed = (int64_t)v.size();
    out->rejected = s->rejected;
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    double sum = 0;
    for (double x : v) sum += x;
    out->mean_ms = v.empty() ? 0 : sum / v.size();
    out->max_ms = v.empty() ? 0 : v.back();
    out->rays_done = s->rays_done;
    const double span = s->t_last - s->t_first;
    out->mrays_s = span > 0 ? s->rays_done / (span * 1e-3) / 1e6 : 0;
    out->batches = s->batches;
    out->mean_batch = s->batches ? (double)s->batch_reqs / s->batches : 0;
    out->max_busy_streams = (int32_t)s->busy_streams_max;
    out->inflight = s->inflight;
    return RF_OK;
}

RF_API rf_status rf_serve_reset_stats(rf_server *s) {
    if (!s) return fail(RF_ERR_INVALID_ARG, "server must not be NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    s->lat_ms.clear();
    s->rays_done = s->rejected = s->batches = s->batch_reqs = s->busy_streams_max = 0;
    s->t_first = -1;
    s->t_last = 0;
    return RF_OK;
}

RF_API rf_status rf_serve_destroy(rf_server *s) {
    if (!s) return RF_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->th.joinable()) s->th.join();
    // launched batches end with a host callback; wait for them before freeing
    for (cudaStream_t st : s->streams) cudaStreamSynchronize(st);
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    cudaFree(s->d_rgb);
    cudaFree(s->d_trans);
    cudaFree(s->d_depth);
    cudaFree(s->d_keys);
    cudaFreeHost(s->h_rgb);
    delete s;
    return RF_OK;
}
