// C-ABI entry points of the encoder (include/fv.h): argument checks, the work
// plan (frames -> statistics row ranges), stream-ordered scratch, and the
// kernel sequence of each precision form:
//
//   FP32 form: f32 posteriors -> f32 statistics -> finalise
//   BF16 form: bf16 convert (FP32 input only) -> fused tcgen05 encoder
//              (posteriors and statistics, gamma kept on chip) -> finalise
//
// Scratch (FP32 posteriors, per-range statistics, the work list, staging copies of
// host inputs/outputs) comes from cudaMallocAsync on the caller's stream and
// goes back with cudaFreeAsync on the same stream, so a call neither
// synchronises the device nor holds memory after its work ends. The pool's
// release threshold is raised once per device so the memory stays cached.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "fv_bf16.h"
#include "fv_internal.h"

namespace fv {

static thread_local std::string t_err;

void set_error(const std::string &msg) { t_err = msg; }
int fail(int status, const std::string &msg) {
    t_err = msg;
    return status;
}
int cuda_fail(cudaError_t e, const char *what) {
    t_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? FV_ERR_OOM : FV_ERR_CUDA;
}

namespace {

// ---- per-device facts ------------------------------------------------------
struct DevFacts {
    int sms = 0;
    bool pool_ready = false;
};
std::mutex g_dev_mu;
DevFacts g_dev[64];

int device_sms(int dev) {
    std::lock_guard<std::mutex> lk(g_dev_mu);
    DevFacts &f = g_dev[dev & 63];
    if (!f.pool_ready) {
        cudaDeviceGetAttribute(&f.sms, cudaDevAttrMultiProcessorCount, dev);
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        f.pool_ready = true;
    }
    return f.sms > 0 ? f.sms : 1;
}

// ---- pinned staging ring for small host->device uploads (work lists) ------
struct StageSlot {
    void *buf = nullptr;
    size_t cap = 0;
    cudaEvent_t ev = nullptr;
    int dev = -1;
};
struct Stage {
    StageSlot slot[4];
    int next = 0;
    ~Stage() {
        for (auto &s : slot) {
            if (s.ev) {
                cudaEventSynchronize(s.ev);
                cudaEventDestroy(s.ev);
            }
            if (s.buf) cudaFreeHost(s.buf);
        }
    }
};
thread_local Stage t_stage;
thread_local uint32_t t_err_word = 0;   // device error word copied back by host-output calls
thread_local std::vector<char> t_wl;      // host image of a call's work list

// Copy `bytes` from host `src` to device `dst` on `st` through a pinned slot.
cudaError_t stage_upload(void *dst, const void *src, size_t bytes, cudaStream_t st) {
    if (bytes == 0) return cudaSuccess;
    int dev = 0;
    cudaGetDevice(&dev);
    StageSlot &s = t_stage.slot[t_stage.next];
    t_stage.next = (t_stage.next + 1) % 4;
    cudaError_t e;
    if (s.ev) {
        if ((e = cudaEventSynchronize(s.ev)) != cudaSuccess) return e;
    }
    if (s.dev != dev && s.ev) {
        cudaEventDestroy(s.ev);
        s.ev = nullptr;
    }
    if (!s.ev) {
        if ((e = cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming)) != cudaSuccess) return e;
        s.dev = dev;
    }
    if (s.cap < bytes) {
        if (s.buf) cudaFreeHost(s.buf);
        s.buf = nullptr;
        s.cap = 0;
        size_t cap = std::max<size_t>(bytes, 1 << 16);
        if ((e = cudaHostAlloc(&s.buf, cap, cudaHostAllocPortable)) != cudaSuccess) return e;
        s.cap = cap;
    }
    std::memcpy(s.buf, src, bytes);
    if ((e = cudaMemcpyAsync(dst, s.buf, bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    return cudaEventRecord(s.ev, st);
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ---- the work plan -----------------------------------------------------------
struct Plan {
    std::vector<FrameInfo> frames;
    std::vector<StatUnit> units;
    std::vector<int2> cta;   // BF16: (first unit, count) per share (one persistent cluster)
    int64_t rows = 0;
    int nonempty = 0;
};

// Split the packed rows into G near-equal shares (boundaries on 128-row
// multiples, the BF16 kernel's tile) and cut each share at frame boundaries:
// every piece is a unit with its own slot. A frame's units come out
// consecutive, in row order.
void make_plan_balanced(const int64_t *offsets, int B, int G, Plan &p);
}  // namespace

void build_balanced_plan(const int64_t *offsets, int B, int G, std::vector<FrameInfo> &frames,
                         std::vector<StatUnit> &units, std::vector<int2> &cta) {
    Plan p;
    make_plan_balanced(offsets, B, G, p);
    frames.swap(p.frames);
    units.swap(p.units);
    cta.swap(p.cta);
}

namespace {
void make_plan_balanced(const int64_t *offsets, int B, int G, Plan &p) {
    p.frames.resize(B);
    p.units.clear();
    p.cta.clear();
    p.rows = offsets[B];
    p.nonempty = 0;
    for (int b = 0; b < B; ++b) {
        p.frames[b].row0 = offsets[b];
        p.frames[b].n = offsets[b + 1] - offsets[b];
        p.frames[b].slot0 = 0;
        p.frames[b].nslots = 0;
        if (p.frames[b].n > 0) ++p.nonempty;
    }
    const int64_t R = p.rows;
    int f = 0;
    int64_t a = 0;
    for (int c = 0; c < G; ++c) {
        const int64_t e = (c == G - 1) ? R : std::max<int64_t>(a, (R * (c + 1) / G) / 128 * 128);
        const int first = (int)p.units.size();
        while (f < B && offsets[f + 1] <= a) ++f;
        for (int ff = f; ff < B && offsets[ff] < e; ++ff) {
            const int64_t s0 = std::max(a, offsets[ff]), s1 = std::min(e, offsets[ff + 1]);
            if (s1 <= s0) continue;
            StatUnit u;
            u.row0 = s0;
            u.nrows = (int32_t)(s1 - s0);
            u.slot = (int32_t)p.units.size();
            if (p.frames[ff].nslots == 0) p.frames[ff].slot0 = u.slot;
            ++p.frames[ff].nslots;
            p.units.push_back(u);
        }
        p.cta.push_back(make_int2(first, (int)p.units.size() - first));
        a = e;
    }
}

// Split every frame into row ranges of at most `rpr` rows; each range becomes
// one statistics unit writing its own slot (the paper's per-block copies).
void make_plan(const int64_t *offsets, int B, int64_t rpr, Plan &p) {
    p.frames.resize(B);
    p.units.clear();
    p.rows = offsets[B];
    int slot = 0;
    for (int b = 0; b < B; ++b) {
        FrameInfo &f = p.frames[b];
        f.row0 = offsets[b];
        f.n = offsets[b + 1] - offsets[b];
        f.slot0 = slot;
        f.nslots = (int32_t)((f.n + rpr - 1) / rpr);
        if (f.n > 0) ++p.nonempty;
        for (int64_t r = 0; r < f.n; r += rpr) {
            StatUnit u;
            u.row0 = f.row0 + r;
            u.nrows = (int32_t)std::min<int64_t>(rpr, f.n - r);
            u.slot = slot++;
            p.units.push_back(u);
        }
    }
}

struct Scratch {
    char *base = nullptr;
    size_t off = 0;
    size_t take(size_t bytes) {
        size_t o = off;
        off += (bytes + 255) / 256 * 256;
        return o;
    }
};

int encode_impl(const fv_gmm *g, const void *X, bool x_bf16, int64_t ld_x, const int64_t *offsets, int B,
                int x_on_device, float *fv_out, int out_on_device, cudaStream_t st, float tau = 0.f,
                unsigned long long *skip_count = nullptr) {
    const int K = g->K, D = g->D, Kp = g->Kp;
    const size_t fvlen = (size_t)2 * K * D;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != g->device) return fail(FV_ERR_INVALID, "GMM handle belongs to another device than the current one");
    if (offsets[0] != 0) return fail(FV_ERR_INVALID, "offsets[0] must be 0");
    for (int b = 0; b < B; ++b)
        if (offsets[b + 1] < offsets[b]) return fail(FV_ERR_INVALID, "offsets must be non-decreasing");
    const int64_t rows = offsets[B];
    if (rows > 0 && !X) return fail(FV_ERR_INVALID, "descriptor pointer is NULL");
    if (x_on_device && X && !is_device_ptr(X)) return fail(FV_ERR_INVALID, "x_on_device=1 but X is not device memory");
    if (out_on_device && !is_device_ptr(fv_out)) return fail(FV_ERR_INVALID, "out_on_device=1 but fv_out is not device memory");

    const int sms = device_sms(g->device);
    const bool bf16 = is_bf16(g->prec);

    Plan plan;
    if (bf16) {
        // persistent clusters over balanced shares of the packed rows
        make_plan_balanced(offsets, B, bf16_shares(g, rows, sms), plan);
    } else {
        // rows per statistics range: aim for about three blocks per SM in one wave
        const int64_t blocks_per_range = (int64_t)(Kp / 64) * ((D + 63) / 64);
        int64_t rpr = (rows * blocks_per_range + 3LL * sms - 1) / (3LL * sms);
        rpr = std::min<int64_t>(std::max<int64_t>(round_up64(rpr, 32), 64), 16384);
        make_plan(offsets, B, rpr, plan);
    }
    const int nslots = (int)plan.units.size();
    const int nctas = (int)plan.cta.size();
    // floats per component in a statistics slot: centred [A|B] blocks of D and S0
    const int P = 2 * D + 1;
    const int64_t ldx_dev = bf16 ? (x_bf16 ? ld_x : (int64_t)g->Dp) : (int64_t)D;

    Scratch s;
    const size_t o_x = (!x_on_device && rows > 0) ? s.take(sizeof(float) * rows * D) : 0;
    const bool need_x_f32_stage = !x_on_device && rows > 0;
    const size_t o_xb = (bf16 && !x_bf16 && rows > 0) ? s.take(sizeof(uint16_t) * rows * ldx_dev) : 0;
    const size_t o_gam = !bf16 ? s.take(f32_gamma_bytes(std::max<int64_t>(rows, 1), Kp)) : 0;
    const size_t o_part = s.take(sizeof(float) * std::max(nslots, 1) * (size_t)Kp * P);
    // the work list (frames, units, shares) and the zeroed error word go up
    // in one staged copy
    const size_t wl_fr = 0;
    const size_t wl_un = round_up64((int64_t)(wl_fr + sizeof(FrameInfo) * B), 16);
    const size_t wl_cta = round_up64((int64_t)(wl_un + sizeof(StatUnit) * std::max(nslots, 1)), 16);
    const size_t wl_err = round_up64((int64_t)(wl_cta + sizeof(int2) * std::max(nctas, 1)), 16);
    const size_t wl_bytes = wl_err + 16;
    const size_t o_wl = s.take(wl_bytes);
    const size_t o_sq = s.take(sizeof(double) * (size_t)B * (Kp / 32) * ((D + 7) / 8));
    const size_t o_out = !out_on_device ? s.take(sizeof(float) * fvlen * B) : 0;
    cudaError_t e = cudaMallocAsync((void **)&s.base, s.off, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(scratch)");

    int rc = FV_OK;
    bool check_err_word = false;
    t_err_word = 0;
    do {
        const void *Xd = X;
        if (need_x_f32_stage) {
            const size_t bytes = x_bf16 ? sizeof(uint16_t) * rows * ld_x : sizeof(float) * rows * D;
            if ((e = cudaMemcpyAsync(s.base + o_x, X, bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess) {
                rc = cuda_fail(e, "cudaMemcpyAsync(X)");
                break;
            }
            Xd = s.base + o_x;
        }
        float *outd = out_on_device ? fv_out : (float *)(s.base + o_out);
        FrameInfo *frd = (FrameInfo *)(s.base + o_wl + wl_fr);
        StatUnit *und = (StatUnit *)(s.base + o_wl + wl_un);
        int2 *ctad = (int2 *)(s.base + o_wl + wl_cta);
        uint32_t *errd = (uint32_t *)(s.base + o_wl + wl_err);
        {
            std::vector<char> &h = t_wl;
            h.assign(wl_bytes, 0);
            std::memcpy(h.data() + wl_fr, plan.frames.data(), sizeof(FrameInfo) * B);
            std::memcpy(h.data() + wl_un, plan.units.data(), sizeof(StatUnit) * nslots);
            std::memcpy(h.data() + wl_cta, plan.cta.data(), sizeof(int2) * nctas);
            if ((e = stage_upload(s.base + o_wl, h.data(), wl_bytes, st)) != cudaSuccess) {
                rc = cuda_fail(e, "work-list upload");
                break;
            }
        }
        float *part = (float *)(s.base + o_part);
        double *sq = (double *)(s.base + o_sq);
        if (!bf16) {
            float *gam = (float *)(s.base + o_gam);
            if ((e = launch_f32_posteriors(g, (const float *)Xd, rows, gam, st)) != cudaSuccess) {
                rc = cuda_fail(e, "f32 posteriors launch");
                break;
            }
            if ((e = launch_f32_stats(g, (const float *)Xd, gam, rows, und, nslots, part, P, st, true, tau, skip_count)) !=
                cudaSuccess) {
                rc = cuda_fail(e, "f32 statistics launch");
                break;
            }
        } else {
            const uint16_t *xb = (const uint16_t *)Xd;
            if (!x_bf16) {
                uint16_t *xconv = (uint16_t *)(s.base + o_xb);
                if ((e = launch_bf16_convert(g, (const float *)Xd, rows, xconv, st)) != cudaSuccess) {
                    rc = cuda_fail(e, "bf16 convert launch");
                    break;
                }
                xb = xconv;
            }
            rc = run_bf16_encoder(g, xb, ldx_dev, rows, und, ctad, nctas, part, P, errd, st, tau, skip_count);
            if (rc != FV_OK) break;
        }
        int max_slots = 1;
        for (const FrameInfo &fi : plan.frames) max_slots = std::max(max_slots, fi.nslots);
        if ((e = launch_finalize(g, part, P, frd, B, sq, outd, st, errd, nullptr, max_slots, true)) !=
            cudaSuccess) {
            rc = cuda_fail(e, "finalise launch");
            break;
        }
        if (!out_on_device) {
            if ((e = cudaMemcpyAsync(fv_out, outd, sizeof(float) * fvlen * B, cudaMemcpyDeviceToHost, st)) !=
                    cudaSuccess ||
                (e = cudaMemcpyAsync(&t_err_word, errd, sizeof(uint32_t), cudaMemcpyDeviceToHost, st)) !=
                    cudaSuccess) {
                rc = cuda_fail(e, "cudaMemcpyAsync(fv_out)");
                break;
            }
            check_err_word = true;
        }
    } while (0);
    cudaError_t ef = cudaFreeAsync(s.base, st);
    if (rc == FV_OK && ef != cudaSuccess) rc = cuda_fail(ef, "cudaFreeAsync(scratch)");
    if (rc == FV_OK && !out_on_device) {
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) rc = cuda_fail(e, "cudaStreamSynchronize");
    }
    if (rc == FV_OK && check_err_word && t_err_word != 0)
        rc = fail(FV_ERR_DEVICE, "a kernel gave up on a bounded wait (error word " + std::to_string(t_err_word) +
                                     "); the output is NaN");
    if (rc == FV_OK && plan.nonempty == 0) rc = fail(FV_ERR_EMPTY, "no descriptors (N == 0)");
    return rc;
}

int check_common(const fv_gmm *g, const void *fv_out) {
    if (!g) return fail(FV_ERR_INVALID, "NULL GMM handle");
    if (!fv_out) return fail(FV_ERR_INVALID, "NULL output pointer");
    return FV_OK;
}

}  // namespace
}  // namespace fv

using namespace fv;

extern "C" const char *fv_last_error(void) { return t_err.c_str(); }

extern "C" int fv_encode(const fv_gmm *gmm, const float *X, int64_t N, int x_on_device, float *fv_out,
                         int out_on_device, void *cuda_stream) {
    int rc = check_common(gmm, fv_out);
    if (rc != FV_OK) return rc;
    if (N < 0) return fail(FV_ERR_INVALID, "N must be >= 0");
    const int64_t offs[2] = {0, N};
    return encode_impl(gmm, X, false, 0, offs, 1, x_on_device, fv_out, out_on_device, (cudaStream_t)cuda_stream);
}

extern "C" int fv_encode_batch(const fv_gmm *gmm, const float *X_packed, const int64_t *offsets, int B,
                               int x_on_device, float *fv_out, int out_on_device, void *cuda_stream) {
    int rc = check_common(gmm, fv_out);
    if (rc != FV_OK) return rc;
    if (B <= 0 || !offsets) return fail(FV_ERR_INVALID, "B must be > 0 and offsets non-NULL");
    return encode_impl(gmm, X_packed, false, 0, offsets, B, x_on_device, fv_out, out_on_device,
                       (cudaStream_t)cuda_stream);
}

extern "C" int fv_encode_batch_bf16(const fv_gmm *gmm, const uint16_t *X_bf16, int64_t ld_x, const int64_t *offsets,
                                    int B, float *fv_out, void *cuda_stream) {
    int rc = check_common(gmm, fv_out);
    if (rc != FV_OK) return rc;
    if (!is_bf16(gmm->prec)) return fail(FV_ERR_INVALID, "fv_encode_batch_bf16 needs an FV_PREC_BF16 or FV_PREC_BF16X2 GMM");
    if (B <= 0 || !offsets) return fail(FV_ERR_INVALID, "B must be > 0 and offsets non-NULL");
    if (ld_x < gmm->D || ld_x % 8 != 0) return fail(FV_ERR_INVALID, "ld_x must be >= D and a multiple of 8");
    if (((uintptr_t)X_bf16) % 16 != 0) return fail(FV_ERR_INVALID, "X_bf16 must be 16-byte aligned");
    return encode_impl(gmm, X_bf16, true, ld_x, offsets, B, 1, fv_out, 1, (cudaStream_t)cuda_stream);
}

extern "C" int fv_encode_batch_opts(const fv_gmm *gmm, const void *X, int x_is_bf16, int64_t ld_x,
                                    const int64_t *offsets, int B, int x_on_device, float *fv_out, int out_on_device,
                                    const fv_encode_options *opts, void *cuda_stream) {
    int rc = check_common(gmm, fv_out);
    if (rc != FV_OK) return rc;
    if (B <= 0 || !offsets) return fail(FV_ERR_INVALID, "B must be > 0 and offsets non-NULL");
    const float tau = opts ? opts->posterior_threshold : 0.f;
    if (!(tau >= 0.f) || !(tau < 1.f)) return fail(FV_ERR_INVALID, "posterior_threshold must be in [0, 1)");
    unsigned long long *cnt = opts ? (unsigned long long *)opts->skip_counts : nullptr;
    if (cnt && !is_device_ptr(cnt)) return fail(FV_ERR_INVALID, "skip_counts must be device memory");
    if (x_is_bf16) {
        if (!is_bf16(gmm->prec)) return fail(FV_ERR_INVALID, "bfloat16 descriptors need an FV_PREC_BF16 GMM");
        if (!x_on_device || !out_on_device)
            return fail(FV_ERR_INVALID, "bfloat16 descriptors and their output must be device memory");
        if (ld_x < gmm->D || ld_x % 8 != 0) return fail(FV_ERR_INVALID, "ld_x must be >= D and a multiple of 8");
        if (((uintptr_t)X) % 16 != 0) return fail(FV_ERR_INVALID, "X must be 16-byte aligned");
        return encode_impl(gmm, X, true, ld_x, offsets, B, 1, fv_out, 1, (cudaStream_t)cuda_stream, tau, cnt);
    }
    return encode_impl(gmm, X, false, 0, offsets, B, x_on_device, fv_out, out_on_device, (cudaStream_t)cuda_stream,
                       tau, cnt);
}

namespace fv {
// fv_encode_pca with the rows either read from X or (yp != nullptr, device
// memory, BF16 form) assembled from a dense-SIFT y-pass buffer.
int encode_pca_impl(const fv_gmm *gmm, const fv_pca *pca, const float *X, const float *xy, const int64_t *offsets,
                    int B, int x_on_device, float *fv_out, int out_on_device, void *cuda_stream, const float *yp,
                    const DsPlan *dsp) {
    int rc = check_common(gmm, fv_out);
    if (rc != FV_OK) return rc;
    if (!pca) return fail(FV_ERR_INVALID, "fv_encode_pca: NULL PCA handle");
    if (B <= 0 || !offsets) return fail(FV_ERR_INVALID, "B must be > 0 and offsets non-NULL");
    int m = 0, Din = 0;
    fv_pca_info(pca, &m, &Din);
    if (gmm->D != m + (xy ? 2 : 0))
        return fail(FV_ERR_INVALID, "fv_encode_pca: the GMM's D must be m + 2 (m without positions)");
    if (offsets[0] != 0) return fail(FV_ERR_INVALID, "offsets[0] must be 0");
    for (int b = 0; b < B; ++b)
        if (offsets[b + 1] < offsets[b]) return fail(FV_ERR_INVALID, "offsets must be non-decreasing");
    const int64_t N = offsets[B];
    if (yp) {
        if (!is_bf16(gmm->prec) || !x_on_device) return fail(FV_ERR_INVALID, "fv_encode_pca: gather needs the BF16 form");
    } else {
        if (N > 0 && !X) return fail(FV_ERR_INVALID, "descriptor pointer is NULL");
        if (x_on_device && N > 0 && (!is_device_ptr(X) || (xy && !is_device_ptr(xy))))
            return fail(FV_ERR_INVALID, "x_on_device=1 but X or xy is not device memory");
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const bool bf16 = is_bf16(gmm->prec);
    const int D = gmm->D, ld = bf16 ? gmm->Dp : D;
    Scratch s;
    const size_t o_x = !x_on_device ? s.take(sizeof(float) * std::max<int64_t>(N, 1) * Din) : 0;
    const size_t o_xy = (!x_on_device && xy) ? s.take(sizeof(float) * 2 * std::max<int64_t>(N, 1)) : 0;
    const size_t o_y = s.take((bf16 ? 2 : 4) * (size_t)std::max<int64_t>(N, 1) * ld);
    const size_t o_err = s.take(16);
    cudaError_t e = cudaMallocAsync((void **)&s.base, s.off, st);
    if (e != cudaSuccess) return cuda_fail(e, "fv_encode_pca: cudaMallocAsync(scratch)");
    const float *Xd = X, *xyd = xy;
    uint32_t *errd = (uint32_t *)(s.base + o_err);
    uint32_t herr = 0;
    do {
        if ((e = cudaMemsetAsync(errd, 0, 4, st)) != cudaSuccess) {
            rc = cuda_fail(e, "fv_encode_pca: memset");
            break;
        }
        if (!x_on_device && N > 0) {
            if ((e = cudaMemcpyAsync(s.base + o_x, X, sizeof(float) * N * Din, cudaMemcpyHostToDevice, st)) !=
                    cudaSuccess ||
                (xy && (e = cudaMemcpyAsync(s.base + o_xy, xy, sizeof(float) * 2 * N, cudaMemcpyHostToDevice, st)) !=
                           cudaSuccess)) {
                rc = cuda_fail(e, "fv_encode_pca: cudaMemcpyAsync(X)");
                break;
            }
            Xd = (const float *)(s.base + o_x);
            xyd = xy ? (const float *)(s.base + o_xy) : nullptr;
        }
        if (!yp && N > 0 && ((uintptr_t)Xd) % 16 != 0) {
            rc = fail(FV_ERR_INVALID, "fv_encode_pca: X must be 16-byte aligned");
            break;
        }
        if ((e = launch_pca(pca, Xd, xyd, N, bf16, s.base + o_y, ld, errd, st, yp, dsp)) != cudaSuccess) {
            rc = cuda_fail(e, "fv_encode_pca: projection launch");
            break;
        }
        rc = encode_impl(gmm, s.base + o_y, bf16, ld, offsets, B, 1, fv_out, out_on_device, st);
        if (rc != FV_OK && rc != FV_ERR_EMPTY) break;
        if (!out_on_device) {
            if ((e = cudaMemcpyAsync(&herr, errd, 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
                (e = cudaStreamSynchronize(st)) != cudaSuccess) {
                rc = cuda_fail(e, "fv_encode_pca: error word");
                break;
            }
            if (herr) rc = fail(FV_ERR_DEVICE, "fv_encode_pca: the projection gave up on a bounded wait");
        }
    } while (0);
    cudaFreeAsync(s.base, st);
    return rc;
}
}  // namespace fv

extern "C" int fv_encode_pca(const fv_gmm *gmm, const fv_pca *pca, const float *X, const float *xy,
                             const int64_t *offsets, int B, int x_on_device, float *fv_out, int out_on_device,
                             void *cuda_stream) {
    return encode_pca_impl(gmm, pca, X, xy, offsets, B, x_on_device, fv_out, out_on_device, cuda_stream, nullptr,
                           nullptr);
}

// ---- instrumentation ------------------------------------------------------------
namespace fv {
namespace {
struct ProfRec {
    std::string name;
    cudaEvent_t a = nullptr, b = nullptr;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof_pending;
std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_prof_free;
std::atomic<int64_t> g_launches{0};
}  // namespace

KernelTimer::KernelTimer(const char *name, cudaStream_t st) : slot_(-1), st_(st) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof_on) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return;   // no event timing inside a graph capture
    }
    ProfRec r;
    r.name = name;
    if (!g_prof_free.empty()) {
        r.a = g_prof_free.back().first;
        r.b = g_prof_free.back().second;
        g_prof_free.pop_back();
    } else {
        if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
    }
    cudaEventRecord(r.a, st);
    g_prof_pending.push_back(r);
    slot_ = (int)g_prof_pending.size() - 1;
}

KernelTimer::~KernelTimer() {
    if (slot_ < 0) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (slot_ < (int)g_prof_pending.size()) cudaEventRecord(g_prof_pending[slot_].b, st_);
}
}  // namespace fv

extern "C" int fv_prof_enable(int on) {
    std::lock_guard<std::mutex> lk(fv::g_prof_mu);
    fv::g_prof_on = on != 0;
    return FV_OK;
}

extern "C" int fv_prof_collect(fv_kernel_stat *out, int max, int *n_out) {
    std::vector<fv::ProfRec> recs;
    {
        std::lock_guard<std::mutex> lk(fv::g_prof_mu);
        recs.swap(fv::g_prof_pending);
    }
    std::vector<fv_kernel_stat> agg;
    int rc = FV_OK;
    for (auto &r : recs) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e != cudaSuccess) rc = fv::cuda_fail(e, "fv_prof_collect");
        size_t i = 0;
        for (; i < agg.size(); ++i)
            if (r.name == agg[i].name) break;
        if (i == agg.size()) {
            fv_kernel_stat s{};
            std::strncpy(s.name, r.name.c_str(), sizeof(s.name) - 1);
            agg.push_back(s);
        }
        agg[i].launches += 1;
        agg[i].total_ms += ms;
    }
    {
        std::lock_guard<std::mutex> lk(fv::g_prof_mu);
        for (auto &r : recs) fv::g_prof_free.emplace_back(r.a, r.b);
    }
    const int n = (int)agg.size();
    if (n_out) *n_out = n;
    for (int i = 0; i < n && i < max && out; ++i) out[i] = agg[i];
    return rc;
}

extern "C" int64_t fv_launch_count(void) { return fv::g_launches.load(); }

namespace fv {
void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace fv
