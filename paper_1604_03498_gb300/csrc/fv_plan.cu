// Batched form: a plan with plan-owned buffers, a measured autotune of the
// statistics grid, and one CUDA graph of the kernel sequence per plan.
//
// The graph is captured once against the plan's buffers: bf16 input rows,
// statistics slots, a device work list and the output vectors. The encoder
// walks the batch's units from the device work list and the finalise takes
// the frame count from its header, and the persistent encoder's grid does not
// depend on the batch, so one capture serves every batch up to the plan's
// capacity. A
// run builds the balanced work list on the host, uploads it (one copy from a
// pinned staging slot) and launches the graph on the caller's stream.
#include <cstdio>
#include <cstring>
#include <fstream>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "fv_bf16.h"
#include "fv_internal.h"

namespace fv {
namespace {

constexpr int kGraphKernels = 4;   // fused encoder, finalise R, A and B

struct WorkHeader {
    int64_t rows;
    int32_t B;
    int32_t pad;
};

// Synthetic bf16 descriptors for timing candidates: a counter-based hash of
// the element index mapped to [-3, 3) (timing only, never a result).
__global__ void synth_fill_kernel(uint16_t *x, int64_t n, uint32_t seed) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t h = (uint32_t)i * 0x9E3779B1u ^ seed;
        h ^= h >> 16;
        h *= 0x7feb352du;
        h ^= h >> 15;
        h *= 0x846ca68bu;
        h ^= h >> 16;
        const float v = (float)(h >> 8) * (6.0f / 16777216.0f) - 3.0f;
        x[i] = (uint16_t)(__float_as_uint(v) >> 16);
    }
}

std::string gpu_key(int dev, int sms, const fv_gmm *g, int64_t max_rows, int max_frames) {
    cudaDeviceProp prop;
    std::string name = "gpu";
    if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) name = prop.name;
    for (auto &ch : name)
        if (ch == ' ' || ch == '|') ch = '_';
    std::ostringstream os;
    os << name << "|" << sms << "|" << g->K << "|" << g->D << "|" << max_rows << "|" << max_frames << "|p" << g->prec;
    return os.str();
}

// Cache lines: key|G|stages (later lines win).
bool read_cache(const char *path, const std::string &key, int *G, int *stages) {
    if (!path) return false;
    std::ifstream f(path);
    std::string line;
    bool found = false;
    while (std::getline(f, line)) {
        if (line.compare(0, key.size(), key) != 0 || line.size() <= key.size() || line[key.size()] != '|') continue;
        int g = 0, st = 0;
        if (std::sscanf(line.c_str() + key.size() + 1, "%d|%d", &g, &st) == 2 && g > 0 && st > 0) {
            *G = g;
            *stages = st;
            found = true;
        }
    }
    return found;
}

void write_cache(const char *path, const std::string &key, int G, int stages) {
    if (!path) return;
    std::ofstream f(path, std::ios::app);
    f << key << "|" << G << "|" << stages << "\n";
}

}  // namespace
}  // namespace fv

using namespace fv;

struct fv_batch_plan {
    const fv_gmm *g = nullptr;
    int device = 0, sms = 1, base = 1, G = 1, Gmax = 1, P = 0, max_frames = 0, max_units = 0;
    int nstage = 0;   // Y stages of the encoder (0: the most that fit)
    int64_t max_rows = 0;
    fv_batch_plan_info info{};
    char *block = nullptr;
    uint16_t *xin = nullptr;
    float *part = nullptr, *out = nullptr;
    double *sq = nullptr;
    uint32_t *err = nullptr;
    char *wl = nullptr;   // device work list: header, frames, units, cta
    size_t wl_bytes = 0, off_frames = 0, off_units = 0, off_cta = 0;
    void *host[2] = {nullptr, nullptr};
    cudaEvent_t ev[2] = {nullptr, nullptr};
    int next = 0;
    cudaGraphExec_t exec = nullptr;
    std::vector<FrameInfo> frames;
    std::vector<StatUnit> units;
    std::vector<int2> cta;
};

namespace fv {
namespace {

// Build the batch's work list for G shares and queue its upload on st.
int upload_work(fv_batch_plan *p, const int64_t *offsets, int B, int G, cudaStream_t st) {
    build_balanced_plan(offsets, B, G, p->frames, p->units, p->cta);
    if ((int)p->units.size() > p->max_units) return fail(FV_ERR_INVALID, "batch plan: work list overflow");
    const int slot = p->next;
    p->next ^= 1;
    cudaError_t e = cudaEventSynchronize(p->ev[slot]);   // previous upload from this slot is done
    if (e != cudaSuccess) return cuda_fail(e, "batch plan: staging event");
    char *h = (char *)p->host[slot];
    std::memset(h, 0, p->wl_bytes);
    WorkHeader hd{offsets[B], B, 0};
    std::memcpy(h, &hd, sizeof(hd));
    std::memcpy(h + p->off_frames, p->frames.data(), sizeof(FrameInfo) * B);
    std::memcpy(h + p->off_units, p->units.data(), sizeof(StatUnit) * p->units.size());
    std::memcpy(h + p->off_cta, p->cta.data(), sizeof(int2) * p->cta.size());
    if ((e = cudaMemcpyAsync(p->wl, h, p->wl_bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaEventRecord(p->ev[slot], st)) != cudaSuccess)
        return cuda_fail(e, "batch plan: work-list upload");
    return FV_OK;
}

// The kernel sequence over the plan's buffers with G statistics shares.
int launch_sequence(fv_batch_plan *p, int G, cudaStream_t st) {
    const fv_gmm *g = p->g;
    cudaError_t e = cudaMemsetAsync(p->err, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return cuda_fail(e, "batch plan: error word");
    const int *B_dev = (const int *)(p->wl + 8);
    int rc = run_bf16_encoder(g, p->xin, g->Dp, p->max_rows, (const StatUnit *)(p->wl + p->off_units),
                              (const int2 *)(p->wl + p->off_cta), G, p->part, p->P, p->err, st, 0.f, nullptr,
                              p->nstage);
    if (rc != FV_OK) return rc;
    if ((e = launch_finalize(g, p->part, p->P, (const FrameInfo *)(p->wl + p->off_frames), p->max_frames, p->sq,
                             p->out, st, p->err, B_dev)) != cudaSuccess)
        return cuda_fail(e, "batch plan: finalise launch");
    return FV_OK;
}

int autotune(fv_batch_plan *p, cudaStream_t st, double *best_ms) {
    // synthetic batch at the plan's capacity: max_frames equal frames
    const int B = p->max_frames;
    std::vector<int64_t> offs(B + 1);
    for (int b = 0; b <= B; ++b) offs[b] = p->max_rows * b / B;
    {
        KernelTimer kt_("synth_fill", st);
        synth_fill_kernel<<<1024, 256, 0, st>>>(p->xin, p->max_rows * p->g->Dp, 20160603u);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "batch plan: synthetic fill");
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const int base = p->base;
    int bestG = base, bestS = bf16_max_stages(p->g);
    *best_ms = 1e30;
    int rc = FV_OK, cands = 0;
    for (int stages = bf16_max_stages(p->g); rc == FV_OK && stages >= 1; --stages) {
        for (int f = 1; rc == FV_OK && f <= 4; ++f) {
            const int G = std::min(p->Gmax, base * f);
            p->nstage = stages;
            float best = 1e30f;
            rc = upload_work(p, offs.data(), B, G, st);
            for (int it = 0; rc == FV_OK && it < 5; ++it) {
                cudaEventRecord(a, st);
                rc = launch_sequence(p, G, st);
                cudaEventRecord(b, st);
                if (rc == FV_OK && cudaEventSynchronize(b) == cudaSuccess && it >= 2) {
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, a, b);
                    best = std::min(best, ms);
                }
            }
            ++cands;
            if (rc == FV_OK && best < *best_ms) {
                *best_ms = best;
                bestG = G;
                bestS = stages;
            }
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (rc != FV_OK) return rc;
    uint32_t errh = 0;
    cudaMemcpy(&errh, p->err, sizeof(errh), cudaMemcpyDeviceToHost);
    if (errh) return fail(FV_ERR_DEVICE, "batch plan: a kernel gave up during the autotune");
    p->G = bestG;
    p->nstage = bestS;
    p->info.candidates = cands;
    return FV_OK;
}

void free_plan(fv_batch_plan *p) {
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    for (int i = 0; i < 2; ++i) {
        if (p->ev[i]) {
            cudaEventSynchronize(p->ev[i]);
            cudaEventDestroy(p->ev[i]);
        }
        if (p->host[i]) cudaFreeHost(p->host[i]);
    }
    if (p->block) cudaFree(p->block);
    delete p;
}

}  // namespace
}  // namespace fv

extern "C" int fv_batch_plan_create(const fv_gmm *gmm, const fv_batch_plan_config *cfg, fv_batch_plan **out) {
    if (!out) return fail(FV_ERR_INVALID, "fv_batch_plan_create: out is NULL");
    *out = nullptr;
    if (!gmm || !cfg) return fail(FV_ERR_INVALID, "fv_batch_plan_create: NULL GMM or config");
    if (!is_bf16(gmm->prec)) return fail(FV_ERR_INVALID, "fv_batch_plan_create: needs an FV_PREC_BF16 or FV_PREC_BF16X2 GMM");
    if (cfg->max_frames < 1 || cfg->max_rows < 1) return fail(FV_ERR_INVALID, "fv_batch_plan_create: empty capacity");
    if (cfg->max_rows > (int64_t)INT32_MAX - 256)
        return fail(FV_ERR_UNSUPPORTED, "fv_batch_plan_create: max_rows beyond 2^31 - 256");
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != gmm->device) return fail(FV_ERR_INVALID, "fv_batch_plan_create: GMM handle on another device");

    fv_batch_plan *p = new fv_batch_plan();
    p->g = gmm;
    p->device = dev;
    cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, dev);
    p->base = bf16_max_shares(gmm, p->sms);
    p->max_frames = cfg->max_frames;
    p->max_rows = cfg->max_rows;
    p->P = 2 * gmm->D + 1;
    p->Gmax = 4 * p->base;
    p->nstage = bf16_max_stages(gmm);
    p->G = p->base;
    p->max_units = p->Gmax + p->max_frames;

    const int Kp = gmm->Kp, Dp = gmm->Dp;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 1023) / 1024 * 1024; return o; };
    const size_t o_x = take(sizeof(uint16_t) * (size_t)p->max_rows * Dp);
    const size_t o_part = take(sizeof(float) * (size_t)p->max_units * Kp * p->P);
    const size_t o_sq = take(sizeof(double) * (size_t)p->max_frames * (Kp / 32) * ((gmm->D + 7) / 8));
    const size_t o_out = take(sizeof(float) * (size_t)p->max_frames * 2 * gmm->K * gmm->D);
    const size_t o_err = take(sizeof(uint32_t));
    p->off_frames = 64;
    p->off_units = p->off_frames + (sizeof(FrameInfo) * p->max_frames + 63) / 64 * 64;
    p->off_cta = p->off_units + (sizeof(StatUnit) * p->max_units + 63) / 64 * 64;
    p->wl_bytes = p->off_cta + sizeof(int2) * p->Gmax;
    const size_t o_wl = take(p->wl_bytes);

    cudaError_t e = cudaMalloc(&p->block, off);
    if (e != cudaSuccess) {
        free_plan(p);
        return fail(FV_ERR_OOM, std::string("fv_batch_plan_create: cudaMalloc: ") + cudaGetErrorString(e));
    }
    p->xin = (uint16_t *)(p->block + o_x);
    p->part = (float *)(p->block + o_part);
    p->sq = (double *)(p->block + o_sq);
    p->out = (float *)(p->block + o_out);
    p->err = (uint32_t *)(p->block + o_err);
    p->wl = p->block + o_wl;
    for (int i = 0; i < 2; ++i) {
        if ((e = cudaHostAlloc(&p->host[i], p->wl_bytes, cudaHostAllocPortable)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&p->ev[i], cudaEventDisableTiming)) != cudaSuccess) {
            free_plan(p);
            return cuda_fail(e, "fv_batch_plan_create: staging");
        }
    }
    cudaStream_t st;
    if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) {
        free_plan(p);
        return cuda_fail(e, "fv_batch_plan_create: stream");
    }
    int rc = FV_OK;
    do {
        // defined contents everywhere: rows past a unit are read (and zeroed)
        // by the encoder's tiles
        if ((e = cudaMemsetAsync(p->block, 0, off, st)) != cudaSuccess) {
            rc = cuda_fail(e, "fv_batch_plan_create: clear");
            break;
        }
        const std::string key = gpu_key(dev, p->sms, gmm, p->max_rows, p->max_frames);
        int cG = 0, cS = 0;
        p->info.tuned = 0;
        if (read_cache(cfg->tune_cache, key, &cG, &cS) && cG <= p->Gmax && cS <= bf16_max_stages(gmm)) {
            p->G = cG;
            p->nstage = cS;
            p->info.tuned = 2;
        } else if (cfg->autotune) {
            double ms = 0.0;
            if ((rc = autotune(p, st, &ms)) != FV_OK) break;
            p->info.tuned = 1;
            p->info.tuned_ms = ms;
            write_cache(cfg->tune_cache, key, p->G, p->nstage);
            cudaMemsetAsync(p->xin, 0, sizeof(uint16_t) * (size_t)p->max_rows * Dp, st);
        }
        // capture the kernel sequence once
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) {
            rc = cuda_fail(e, "fv_batch_plan_create: sync");
            break;
        }
        cudaGraph_t graph = nullptr;
        if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed)) != cudaSuccess) {
            rc = cuda_fail(e, "fv_batch_plan_create: begin capture");
            break;
        }
        rc = launch_sequence(p, p->G, st);
        e = cudaStreamEndCapture(st, &graph);
        if (rc != FV_OK) {
            if (graph) cudaGraphDestroy(graph);
            break;
        }
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "fv_batch_plan_create: end capture");
            break;
        }
        e = cudaGraphInstantiate(&p->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "fv_batch_plan_create: instantiate");
            break;
        }
    } while (0);
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    if (rc != FV_OK) {
        free_plan(p);
        return rc;
    }
    p->info.stat_ctas = p->G;
    p->info.max_rows = p->max_rows;
    p->info.max_frames = p->max_frames;
    p->info.ld_x = gmm->Dp;
    p->info.rows_per_tile = 128;
    p->info.y_stages = p->nstage;
    p->info.tiles_per_share = (double)((p->max_rows + 127) / 128) / p->G;
    *out = p;
    return FV_OK;
}

extern "C" int fv_batch_plan_buffers(fv_batch_plan *p, uint16_t **x_bf16, float **fv_out) {
    if (!p) return fail(FV_ERR_INVALID, "fv_batch_plan_buffers: NULL plan");
    if (x_bf16) *x_bf16 = p->xin;
    if (fv_out) *fv_out = p->out;
    return FV_OK;
}

extern "C" int fv_batch_plan_get_info(const fv_batch_plan *p, fv_batch_plan_info *info) {
    if (!p || !info) return fail(FV_ERR_INVALID, "fv_batch_plan_get_info: NULL argument");
    *info = p->info;
    return FV_OK;
}

static int check_offsets(const fv_batch_plan *p, const int64_t *offsets, int B) {
    if (!offsets || B < 1 || B > p->max_frames) return fail(FV_ERR_INVALID, "batch plan: B outside 1..max_frames");
    if (offsets[0] != 0) return fail(FV_ERR_INVALID, "batch plan: offsets[0] must be 0");
    for (int b = 0; b < B; ++b)
        if (offsets[b + 1] < offsets[b]) return fail(FV_ERR_INVALID, "batch plan: offsets must be non-decreasing");
    if (offsets[B] > p->max_rows) return fail(FV_ERR_INVALID, "batch plan: batch exceeds max_rows");
    return FV_OK;
}

extern "C" int fv_batch_plan_run(fv_batch_plan *p, const int64_t *offsets, int B, float *fv_out, int out_on_device,
                                 void *cuda_stream) {
    if (!p) return fail(FV_ERR_INVALID, "fv_batch_plan_run: NULL plan");
    int rc = check_offsets(p, offsets, B);
    if (rc != FV_OK) return rc;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if ((rc = upload_work(p, offsets, B, p->G, st)) != FV_OK) return rc;
    cudaError_t e = cudaGraphLaunch(p->exec, st);
    if (e != cudaSuccess) return cuda_fail(e, "fv_batch_plan_run: graph launch");
    count_launches(kGraphKernels);
    if (fv_out) {
        const size_t bytes = sizeof(float) * (size_t)B * 2 * p->g->K * p->g->D;
        if ((e = cudaMemcpyAsync(fv_out, p->out, bytes, out_on_device ? cudaMemcpyDeviceToDevice
                                                                      : cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return cuda_fail(e, "fv_batch_plan_run: output copy");
        if (!out_on_device) {
            uint32_t errh = 0;
            if ((e = cudaMemcpyAsync(&errh, p->err, sizeof(errh), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
                (e = cudaStreamSynchronize(st)) != cudaSuccess)
                return cuda_fail(e, "fv_batch_plan_run: synchronise");
            if (errh) return fail(FV_ERR_DEVICE, "fv_batch_plan_run: a kernel gave up on a bounded wait");
        }
    }
    return offsets[B] > 0 ? FV_OK : fail(FV_ERR_EMPTY, "no descriptors (N == 0)");
}

extern "C" int fv_batch_plan_run_f32(fv_batch_plan *p, const float *X, const int64_t *offsets, int B, float *fv_out,
                                     int out_on_device, void *cuda_stream) {
    if (!p) return fail(FV_ERR_INVALID, "fv_batch_plan_run_f32: NULL plan");
    int rc = check_offsets(p, offsets, B);
    if (rc != FV_OK) return rc;
    if (offsets[B] > 0 && !X) return fail(FV_ERR_INVALID, "fv_batch_plan_run_f32: NULL descriptors");
    cudaError_t e = launch_bf16_convert(p->g, X, offsets[B], p->xin, (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) return cuda_fail(e, "fv_batch_plan_run_f32: convert");
    return fv_batch_plan_run(p, offsets, B, fv_out, out_on_device, cuda_stream);
}

extern "C" int fv_batch_plan_load_bf16(fv_batch_plan *p, const uint16_t *X, int64_t ld_x, int64_t rows,
                                       void *cuda_stream) {
    if (!p) return fail(FV_ERR_INVALID, "fv_batch_plan_load_bf16: NULL plan");
    if (rows < 0 || rows > p->max_rows) return fail(FV_ERR_INVALID, "fv_batch_plan_load_bf16: rows outside capacity");
    if (ld_x < p->g->D) return fail(FV_ERR_INVALID, "fv_batch_plan_load_bf16: ld_x < D");
    if (rows == 0) return FV_OK;
    cudaError_t e = cudaMemcpy2DAsync(p->xin, sizeof(uint16_t) * p->g->Dp, X, sizeof(uint16_t) * ld_x,
                                      sizeof(uint16_t) * p->g->D, (size_t)rows, cudaMemcpyDeviceToDevice,
                                      (cudaStream_t)cuda_stream);
    return e == cudaSuccess ? FV_OK : cuda_fail(e, "fv_batch_plan_load_bf16: copy");
}

extern "C" void fv_batch_plan_destroy(fv_batch_plan *p) {
    if (!p) return;
    int cur = 0;
    cudaGetDevice(&cur);
    const int dev = p->device;
    if (cur != dev) cudaSetDevice(dev);
    fv::free_plan(p);
    if (cur != dev) cudaSetDevice(cur);
}
