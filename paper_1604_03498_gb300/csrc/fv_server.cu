// Serving form: continuous batching of frames from many video streams.
//
// Client threads submit frames as they arrive. Admission is by device memory:
// a frame is taken only while the descriptors of admitted, unfinished frames
// fit in the HBM budget and a slot is free; otherwise the caller gets
// FV_ERR_BUSY at once and retries. Admitted frames are copied to device memory
// (stream-ordered pool allocations) before submit returns.
//
// One scheduler thread forms batches from the admitted frames in arrival
// order and alternates two batch plans on two streams: while one plan's graph
// runs, the next batch is packed and launched on the other, so frames that
// arrive while the GPU is busy are admitted into the next batch and their
// work overlaps with the batch in flight. One kernel reads every frame of a
// batch from its own device buffer and writes the plan's bfloat16 input rows
// (no packed FP32 copy in between). A host callback enqueued behind
// each batch's result copy stamps the completion time and wakes pollers.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_bf16.h>

#include "fv_internal.h"

namespace fv {
namespace {

// The batch's input in one pass: frame b's FP32 rows, still in the request's
// own device buffer src[b], are rounded to bfloat16 and stored at rows
// off[b] .. off[b+1]-1 of the plan's input (row pitch Dp, columns past D
// zero). Grid (x, B): blockIdx.y is the frame, the x blocks stride over its
// rows.
__global__ void gather_convert_kernel(const float *const *__restrict__ src, const int64_t *__restrict__ off, int D,
                                      int Dp, uint16_t *__restrict__ Xb) {
    const int b = blockIdx.y;
    const float *x = src[b];
    const int64_t r0 = off[b], n = (off[b + 1] - r0) * Dp;
    uint16_t *dst = Xb + r0 * Dp;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / Dp;
        const int d = (int)(i - r * Dp);
        __nv_bfloat16 h = __float2bfloat16_rn(d < D ? x[r * D + d] : 0.f);
        dst[i] = *reinterpret_cast<uint16_t *>(&h);
    }
}

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Request {
    uint64_t ticket = 0;
    int stream_id = 0;
    int64_t n = 0;
    size_t bytes = 0;
    float *dev = nullptr;
    int64_t t_submit = 0, t_launch = 0, t_done = 0;
    int status = FV_PENDING;
    int batch_frames = 0;
    bool done = false;
    std::vector<float> result;
};

}  // namespace
}  // namespace fv

using namespace fv;

struct fv_server {
    const fv_gmm *g = nullptr;
    fv_server_config cfg{};
    int device = 0;
    size_t fvlen = 0;
    fv_batch_plan *plan[2] = {nullptr, nullptr};
    cudaStream_t stream[2] = {nullptr, nullptr};
    uint16_t *xin[2] = {nullptr, nullptr};    // the plans' bf16 input rows (device, owned by the plans)
    void *table_h[2] = {nullptr, nullptr};    // a batch's source pointers and row offsets (pinned)
    void *table_d[2] = {nullptr, nullptr};    // their device copy, read by the gather-convert kernel
    float *plan_out[2] = {nullptr, nullptr};  // plan output buffers (device)
    float *host_out[2] = {nullptr, nullptr};  // pinned copies of a batch's vectors
    std::vector<Request *> batch_reqs[2];
    bool busy[2] = {false, false};
    cudaStream_t copy_stream = nullptr;

    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::deque<Request *> pending;
    std::unordered_map<uint64_t, Request *> tickets;
    int64_t admitted_bytes = 0;
    int64_t pending_rows = 0;
    int slots_used = 0;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread sched;
    int64_t n_admitted = 0, n_refused = 0, n_completed = 0, n_batches = 0;
};

namespace fv {
namespace {

struct DoneArg {
    fv_server *s;
    int i;
};

// Runs on a CUDA callback thread once a batch's vectors are on the host; it
// makes no CUDA calls.
void CUDART_CB on_batch_done(void *arg) {
    DoneArg *a = static_cast<DoneArg *>(arg);
    fv_server *s = a->s;
    const int i = a->i;
    delete a;
    const int64_t t = now_ns();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto &reqs = s->batch_reqs[i];
        for (size_t b = 0; b < reqs.size(); ++b) {
            Request *r = reqs[b];
            const float *src = s->host_out[i] + b * s->fvlen;
            r->result.assign(src, src + s->fvlen);
            r->status = (s->fvlen > 0 && src[0] != src[0]) ? FV_ERR_DEVICE : FV_OK;   // NaN-poisoned batch
            r->t_done = t;
            r->batch_frames = (int)reqs.size();
            r->done = true;
            s->admitted_bytes -= (int64_t)r->bytes;
        }
        s->n_completed += (int64_t)reqs.size();
        reqs.clear();
        s->busy[i] = false;
    }
    s->cv_done.notify_all();
    s->cv_sched.notify_one();
}

size_t table_bytes(int max_frames) { return sizeof(float *) * max_frames + sizeof(int64_t) * (max_frames + 1); }

// Uploads the batch's table (pinned; not rewritten before stream i's batch
// completes) and converts every frame straight into the plan's input.
int gather(fv_server *s, int i, int B, int64_t maxn) {
    const cudaStream_t st = s->stream[i];
    const int maxf = s->cfg.max_batch_frames;
    cudaError_t e = cudaMemcpyAsync(s->table_d[i], s->table_h[i], table_bytes(maxf), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "fv_server: table upload");
    const int Dp = s->g->Dp;
    const int64_t per_frame = (maxn * Dp + 255) / 256;
    const int gx = (int)std::max<int64_t>(1, std::min<int64_t>(per_frame, std::max(1, 8192 / B)));
    const float *const *srcs = static_cast<const float *const *>(s->table_d[i]);
    {
        KernelTimer kt_("gather_convert", st);
        gather_convert_kernel<<<dim3(gx, B), 256, 0, st>>>(srcs, reinterpret_cast<const int64_t *>(srcs + maxf),
                                                           s->g->D, Dp, s->xin[i]);
    }
    e = cudaGetLastError();
    return e == cudaSuccess ? FV_OK : cuda_fail(e, "fv_server: gather-convert launch");
}

void scheduler(fv_server *s) {
    cudaSetDevice(s->device);
    std::vector<int64_t> offs;
    while (true) {
        int i = -1;
        std::vector<Request *> take;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            // launch when a plan is free and the pending frames fill a batch or
            // the oldest has waited batch_window_ns
            while (true) {
                if (s->stop) break;
                if (!s->pending.empty() && (!s->busy[0] || !s->busy[1])) {
                    const bool full = (int)s->pending.size() >= s->cfg.max_batch_frames ||
                                      s->pending_rows >= s->cfg.max_batch_descriptors;
                    const int64_t deadline = s->pending.front()->t_submit + s->cfg.batch_window_ns;
                    const int64_t now = now_ns();
                    if (full || s->cfg.batch_window_ns <= 0 || now >= deadline) break;
                    s->cv_sched.wait_for(lk, std::chrono::nanoseconds(deadline - now));
                } else {
                    s->cv_sched.wait(lk);
                }
            }
            if (s->stop && (s->pending.empty() || (s->busy[0] && s->busy[1]))) break;
            i = !s->busy[0] ? 0 : 1;
            int64_t rows = 0;
            while (!s->pending.empty() && (int)take.size() < s->cfg.max_batch_frames) {
                Request *r = s->pending.front();
                if (rows + r->n > s->cfg.max_batch_descriptors && !take.empty()) break;
                rows += r->n;
                take.push_back(r);
                s->pending.pop_front();
                s->pending_rows -= r->n;
            }
            s->busy[i] = true;
            s->batch_reqs[i] = take;
            ++s->n_batches;
        }
        // gather the frames into the plan's input, encode, copy back; every step ordered on stream i
        const int B = (int)take.size();
        offs.assign(B + 1, 0);
        const int64_t t = now_ns();
        const float **srcs = static_cast<const float **>(s->table_h[i]);
        int64_t maxn = 0;
        for (int b = 0; b < B; ++b) {
            Request *r = take[b];
            r->t_launch = t;
            offs[b + 1] = offs[b] + r->n;
            srcs[b] = r->dev;
            maxn = std::max(maxn, r->n);
        }
        std::memcpy(reinterpret_cast<int64_t *>(srcs + s->cfg.max_batch_frames), offs.data(), sizeof(int64_t) * (B + 1));
        int rc = gather(s, i, B, maxn);
        for (Request *r : take) {   // stream-ordered: freed once the gather has read them
            cudaFreeAsync(r->dev, s->stream[i]);
            r->dev = nullptr;
        }
        if (rc == FV_OK) rc = fv_batch_plan_run(s->plan[i], offs.data(), B, nullptr, 1, s->stream[i]);
        if (rc == FV_OK &&
            cudaMemcpyAsync(s->host_out[i], s->plan_out[i], sizeof(float) * s->fvlen * take.size(),
                            cudaMemcpyDeviceToHost, s->stream[i]) != cudaSuccess)
            rc = FV_ERR_CUDA;
        if (rc == FV_OK && cudaLaunchHostFunc(s->stream[i], on_batch_done, new DoneArg{s, i}) != cudaSuccess)
            rc = FV_ERR_CUDA;
        if (rc != FV_OK) {   // complete the batch's frames with the error
            cudaGetLastError();
            cudaStreamSynchronize(s->stream[i]);
            std::lock_guard<std::mutex> lk(s->mu);
            for (Request *r : take) {
                r->status = rc;
                r->t_done = now_ns();
                r->done = true;
                s->admitted_bytes -= (int64_t)r->bytes;
            }
            s->batch_reqs[i].clear();
            s->busy[i] = false;
            s->cv_done.notify_all();
        }
    }
}

void destroy_server(fv_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_sched.notify_all();
    if (s->sched.joinable()) s->sched.join();
    for (int i = 0; i < 2; ++i)
        if (s->stream[i]) cudaStreamSynchronize(s->stream[i]);
    // every request (pending, in a finished batch, or completed and not yet
    // polled) is in the ticket map exactly once
    for (auto &kv : s->tickets) {
        if (kv.second->dev) cudaFree(kv.second->dev);
        delete kv.second;
    }
    s->tickets.clear();
    s->pending.clear();
    for (int i = 0; i < 2; ++i) {
        if (s->plan[i]) fv_batch_plan_destroy(s->plan[i]);
        if (s->table_h[i]) cudaFreeHost(s->table_h[i]);
        if (s->table_d[i]) cudaFree(s->table_d[i]);
        if (s->host_out[i]) cudaFreeHost(s->host_out[i]);
        if (s->stream[i]) cudaStreamDestroy(s->stream[i]);
    }
    if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
    delete s;
}

}  // namespace
}  // namespace fv

extern "C" int fv_server_create(const fv_gmm *gmm, const fv_server_config *cfg, fv_server **out) {
    if (!out) return fail(FV_ERR_INVALID, "fv_server_create: out is NULL");
    *out = nullptr;
    if (!gmm || !cfg) return fail(FV_ERR_INVALID, "fv_server_create: NULL GMM or config");
    if (!is_bf16(gmm->prec)) return fail(FV_ERR_INVALID, "fv_server_create: needs an FV_PREC_BF16 or FV_PREC_BF16X2 GMM");
    if (cfg->max_slots < 1 || cfg->hbm_budget_bytes <= 0 || cfg->max_batch_frames < 1 ||
        cfg->max_batch_frames > 65535 ||
        cfg->max_frame_descriptors < 1 || cfg->max_batch_descriptors < cfg->max_frame_descriptors)
        return fail(FV_ERR_INVALID, "fv_server_create: inconsistent configuration");
    fv_server *s = new fv_server();
    s->g = gmm;
    s->cfg = *cfg;
    s->fvlen = (size_t)2 * gmm->K * gmm->D;
    cudaGetDevice(&s->device);
    int rc = FV_OK;
    cudaError_t e;
    do {
        if ((e = cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking)) != cudaSuccess) {
            rc = cuda_fail(e, "fv_server_create: stream");
            break;
        }
        for (int i = 0; i < 2 && rc == FV_OK; ++i) {
            fv_batch_plan_config pc{cfg->max_batch_frames, cfg->max_batch_descriptors, 0, nullptr};
            if ((rc = fv_batch_plan_create(gmm, &pc, &s->plan[i])) != FV_OK) break;
            fv_batch_plan_buffers(s->plan[i], &s->xin[i], &s->plan_out[i]);
            if ((e = cudaStreamCreateWithFlags(&s->stream[i], cudaStreamNonBlocking)) != cudaSuccess ||
                (e = cudaHostAlloc(&s->table_h[i], table_bytes(cfg->max_batch_frames), cudaHostAllocPortable)) !=
                    cudaSuccess ||
                (e = cudaMalloc(&s->table_d[i], table_bytes(cfg->max_batch_frames))) != cudaSuccess ||
                (e = cudaHostAlloc(&s->host_out[i], sizeof(float) * s->fvlen * cfg->max_batch_frames,
                                   cudaHostAllocPortable)) != cudaSuccess)
                rc = cuda_fail(e, "fv_server_create: buffers");
        }
    } while (0);
    if (rc != FV_OK) {
        destroy_server(s);
        return rc;
    }
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, s->device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    s->sched = std::thread(scheduler, s);
    *out = s;
    return FV_OK;
}

extern "C" int fv_server_submit(fv_server *s, int stream_id, const float *X, int64_t N, uint64_t *ticket) {
    if (!s || !X || !ticket) return fail(FV_ERR_INVALID, "fv_server_submit: NULL argument");
    if (N < 1 || N > s->cfg.max_frame_descriptors)
        return fail(FV_ERR_INVALID, "fv_server_submit: N outside 1..max_frame_descriptors");
    const size_t bytes = sizeof(float) * (size_t)N * s->g->D;
    Request *r = new Request();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) {
            delete r;
            return fail(FV_ERR_INVALID, "fv_server_submit: server is shutting down");
        }
        if (s->slots_used >= s->cfg.max_slots || s->admitted_bytes + (int64_t)bytes > s->cfg.hbm_budget_bytes) {
            ++s->n_refused;
            delete r;
            return fail(FV_ERR_BUSY, "fv_server_submit: admission refused (slots or HBM budget)");
        }
        s->admitted_bytes += (int64_t)bytes;
        ++s->slots_used;
        ++s->n_admitted;
        r->ticket = s->next_ticket++;
    }
    r->stream_id = stream_id;
    r->n = N;
    r->bytes = bytes;
    r->t_submit = now_ns();
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != s->device) cudaSetDevice(s->device);
    cudaEvent_t ev = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&r->dev, bytes, s->copy_stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(r->dev, X, bytes, cudaMemcpyHostToDevice, s->copy_stream);
    if (e == cudaSuccess) e = cudaEventRecord(ev, s->copy_stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev);   // X may be reused once submit returns
    if (ev) cudaEventDestroy(ev);
    if (cur != s->device) cudaSetDevice(cur);
    if (e != cudaSuccess) {
        if (r->dev) cudaFreeAsync(r->dev, s->copy_stream);
        std::lock_guard<std::mutex> lk(s->mu);
        s->admitted_bytes -= (int64_t)bytes;
        --s->slots_used;
        delete r;
        return cuda_fail(e, "fv_server_submit: copy");
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->tickets[r->ticket] = r;
        s->pending.push_back(r);
        s->pending_rows += r->n;
    }
    s->cv_sched.notify_one();
    *ticket = r->ticket;
    return FV_OK;
}

extern "C" int fv_server_poll(fv_server *s, uint64_t ticket, float *fv_out, fv_result_info *info, int64_t timeout_ns) {
    if (!s) return fail(FV_ERR_INVALID, "fv_server_poll: NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return fail(FV_ERR_NOTFOUND, "fv_server_poll: unknown ticket");
    Request *r = it->second;
    if (!r->done && timeout_ns != 0) {
        auto pred = [&] { return r->done; };
        if (timeout_ns < 0)
            s->cv_done.wait(lk, pred);
        else
            s->cv_done.wait_for(lk, std::chrono::nanoseconds(timeout_ns), pred);
    }
    if (!r->done) return timeout_ns == 0 ? FV_PENDING : fail(FV_ERR_TIMEOUT, "fv_server_poll: wait expired");
    if (fv_out && r->status == FV_OK) std::memcpy(fv_out, r->result.data(), sizeof(float) * s->fvlen);
    if (info) {
        info->status = r->status;
        info->stream_id = r->stream_id;
        info->n = r->n;
        info->latency_ns = r->t_done - r->t_submit;
        info->queue_ns = r->t_launch - r->t_submit;
        info->batch_frames = r->batch_frames;
    }
    const int st = r->status;
    s->tickets.erase(it);
    --s->slots_used;
    delete r;
    return st == FV_OK ? FV_OK : fail(st, "fv_server_poll: the frame's batch failed");
}

extern "C" int fv_server_stats(const fv_server *s, int64_t *admitted, int64_t *refused, int64_t *completed,
                               int64_t *batches) {
    if (!s) return fail(FV_ERR_INVALID, "fv_server_stats: NULL server");
    fv_server *m = const_cast<fv_server *>(s);
    std::lock_guard<std::mutex> lk(m->mu);
    if (admitted) *admitted = s->n_admitted;
    if (refused) *refused = s->n_refused;
    if (completed) *completed = s->n_completed;
    if (batches) *batches = s->n_batches;
    return FV_OK;
}

extern "C" void fv_server_destroy(fv_server *s) {
    if (!s) return;
    int cur = 0;
    cudaGetDevice(&cur);
    const int dev = s->device;
    if (cur != dev) cudaSetDevice(dev);
    fv::destroy_server(s);
    if (cur != dev) cudaSetDevice(cur);
}
