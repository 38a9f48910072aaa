// spl_api.cu -- the C ABI (include/splotch.h): context, particle storage,
// camera / colour map / parameters, and the per-frame pipeline
//   raster+count -> count large -> scan -> [sync: size lists] -> scatter ->
//   tile pass -> large pass -> (E=A epilogue)
// all on one stream.
#include <cmath>
#include <cstdio>
#include <cstddef>
#include <cstring>
#include <new>

#include "splotch.h"
#include "spl_internal.cuh"

using namespace spl;

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

template <typename T>
struct DevBuf {
    T *p = nullptr;
    size_t cap = 0;   // elements
    int ensure(size_t n) {
        if (n <= cap && p) return SPL_OK;
        size_t want = n < 16 ? 16 : n + n / 4;
        T *q = nullptr;
        if (cudaMalloc((void **)&q, want * sizeof(T)) != cudaSuccess) {
            cudaGetLastError();
            return SPL_ENOMEM;
        }
        if (p) cudaFree(p);
        p = q;
        cap = want;
        return SPL_OK;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
};

struct spl_ctx {
    int device = 0;
    int sms = 1;
    cudaStream_t stream = nullptr;
    // particles (SoA)
    int64_t n = 0;
    int attr_type = SPL_ATTR_F32;
    float h_log2_min = 0.f;            // SPL_ATTR_LOGH16
    bool have_particles = false;
    DevBuf<float> x, y, z;
    DevBuf<unsigned char> h, I, s;
    DevBuf<float> cr, cg, cb;          // optional colour components
    bool have_rgb = false;
    // out-of-core rendering (spl_render_stream): two device chunks, filled on
    // a copy stream; while a chunk renders, the pipeline reads it instead of
    // the loaded SoA and adds into the image
    DevBuf<float> cx[2], cy[2], cz[2];
    DevBuf<unsigned char> ch[2], cI[2], cs[2];
    DevBuf<float> ccr[2], ccg[2], ccb[2];
    bool chunk_rgb = false;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t copied[2] = {}, consumed[2] = {};
    bool streaming = false;
    int chunk_buf = 0;
    int64_t chunk_n = 0;
    int chunk_attr = SPL_ATTR_F32;
    float chunk_h_log2_min = 0.f;
    bool accumulate = false;      // the image already holds earlier chunks
    bool last_chunk = true;       // apply the E=A map after this render
    // colour map
    DevBuf<float> pal;
    int npal = 0;
    float s_min = 0.f, s_max = 1.f;
    // camera and parameters
    spl_camera cam{};
    bool have_cam = false;
    spl_params par{};
    // scratch
    DevBuf<Rec> recs;
    // absorption mode: (A, depth key) per record, the depth-order sort, and the
    // (C, T) partials of split tiles
    DevBuf<float2> rec2;
    DevBuf<unsigned long long> pkeys, ptmp, ekeys, etmp;
    DevBuf<unsigned> rank;
    DevBuf<int> sort_hist;
    DevBuf<float4> partial;
    DevBuf<int> counts, ovf;
    DevBuf<int2> ctab;
    DevBuf<long long> offsets, cursor;
    DevBuf<unsigned> large_ids, entries;
    DevBuf<int> item_counts, item_offsets;
    DevBuf<WorkItem> items;
    DevBuf<DevStats> dstats;
    DevBuf<float> host_img_scratch;
    DevStats *hstats = nullptr;   // pinned
    // views of the current batch: constants and image pointers, staged in
    // pinned memory and copied to the device by every render (also inside a
    // captured graph, where the copies read the staging at replay time)
    DevBuf<FrameConst> d_fcs;
    DevBuf<float *> d_images;
    FrameConst *h_fcs = nullptr;  // pinned, kMaxViews
    float **h_images = nullptr;   // pinned, kMaxViews
    // CUDA graph of the batch pipeline (spl_render_batch)
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    unsigned long long graph_key = 0;   // configuration the graph was captured for
    int graph_kernels = 0;              // kernel nodes of the captured graph
    unsigned long long buf_gen = 0;     // bumped whenever a scratch buffer moves
    bool use_graph = true;
    // scheduling of the work items, and the per-item samples that train it
    DevBuf<float> feat, cost, theta, heur;
    DevBuf<int> item_n, order, order_hist;
    DevBuf<long long> item_cycles;
    bool have_model = false;
    bool recording = false;
    int last_items = 0;                 // work items of the last eager render
    // timing: two event sets, so that a frame's stage times are read at the
    // next frame's synchronisation point without an extra wait
    bool timing = false;
    cudaEvent_t stats_ready = nullptr;  // binning counts copied to hstats
    cudaEvent_t ev[2][6] = {};
    int ev_set = 0;
    bool ev_pending[2] = {false, false};
    double sum_ms[6] = {};
    int64_t timed_frames = 0;
    float last_ms[6] = {};
    spl_stats last{};
};

thread_local long long spl::g_launches = 0;

static int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return SPL_OK;
    if (e == cudaErrorMemoryAllocation) return SPL_ENOMEM;
    return SPL_ECUDA;
}

#define SPL_TRY(expr)                      \
    do {                                   \
        int _rc = (expr);                  \
        if (_rc != SPL_OK) return _rc;     \
    } while (0)
#define SPL_CUDA(expr) SPL_TRY(cuda_status(expr))

extern "C" const char *spl_error_string(int code) {
    switch (code) {
        case SPL_OK: return "ok";
        case SPL_EINVAL: return "invalid argument";
        case SPL_ENOMEM: return "out of memory";
        case SPL_ECUDA: return "CUDA error";
        case SPL_ESTATE: return "call out of order";
        case SPL_EDEVICE: return "device-side check failed";
        case SPL_ELIMIT: return "size beyond the fixed scratch of spl_render_noalloc";
        default: return "unknown status";
    }
}

extern "C" int spl_default_params(spl_params *q) {
    if (!q) return SPL_EINVAL;
    q->chi = 3.0;
    q->sigma_per_h = 1.0;
    q->s_box = 1.0;
    q->r_sml = 0.5;
    q->brightness = 1.0;
    q->tile_px = 32;
    q->r_small = 2.0;
    q->r_large = 64.0;
    q->mode = SPL_MODE_ADDITIVE;
    q->sched = SPL_SCHED_NONE;
    q->absorption = 1.0;
    q->log_flags = 0;
    return SPL_OK;
}

static bool params_ok(const spl_params *q) {
    return q && std::isfinite(q->chi) && q->chi > 0 && std::isfinite(q->sigma_per_h) &&
           q->sigma_per_h > 0 && std::isfinite(q->s_box) && q->s_box > 0 &&
           std::isfinite(q->r_sml) && q->r_sml >= 0 && std::isfinite(q->brightness) &&
           (q->tile_px == 16 || q->tile_px == 32 || q->tile_px == 64) && std::isfinite(q->r_small) &&
           q->r_small >= q->r_sml && std::isfinite(q->r_large) && q->r_large >= q->r_small &&
           (q->mode == SPL_MODE_ADDITIVE || q->mode == SPL_MODE_EA || q->mode == SPL_MODE_ABSORB) &&
           q->sched >= 0 && q->sched <= SPL_SCHED_MLP && std::isfinite(q->absorption) &&
           q->absorption > 0 && q->log_flags >= 0 && q->log_flags <= (SPL_LOG_I | SPL_LOG_S);
}

static bool camera_ok(const spl_camera *c) {
    if (!c) return false;
    if (c->width < 1 || c->height < 1 || c->width > 16384 || c->height > 16384) return false;
    if (!(c->fov_y_deg > 0 && c->fov_y_deg < 180) || !(c->z_near > 0)) return false;
    double f[3], r[3];
    for (int k = 0; k < 3; ++k) {
        if (!std::isfinite(c->eye[k]) || !std::isfinite(c->target[k]) || !std::isfinite(c->up[k]))
            return false;
        f[k] = c->target[k] - c->eye[k];
    }
    r[0] = f[1] * c->up[2] - f[2] * c->up[1];
    r[1] = f[2] * c->up[0] - f[0] * c->up[2];
    r[2] = f[0] * c->up[1] - f[1] * c->up[0];
    return (f[0] * f[0] + f[1] * f[1] + f[2] * f[2]) > 0 && (r[0] * r[0] + r[1] * r[1] + r[2] * r[2]) > 0;
}

extern "C" int spl_create(spl_ctx **out, int device, void *stream) {
    if (!out) return SPL_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        return SPL_ECUDA;
    }
    if (device < 0 || device >= ndev) return SPL_EINVAL;
    DeviceGuard g(device);
    spl_ctx *c = new (std::nothrow) spl_ctx();
    if (!c) return SPL_ENOMEM;
    c->device = device;
    c->stream = (cudaStream_t)stream;
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
    spl_default_params(&c->par);
    int rc = c->dstats.ensure(1);
    if (rc == SPL_OK && cudaMemset(c->dstats.p, 0, sizeof(DevStats)) != cudaSuccess) rc = SPL_ECUDA;
    if (rc == SPL_OK && cudaMallocHost((void **)&c->hstats, sizeof(DevStats)) != cudaSuccess)
        rc = SPL_ENOMEM;
    if (rc == SPL_OK && cudaMallocHost((void **)&c->h_fcs, sizeof(FrameConst) * kMaxViews) != cudaSuccess)
        rc = SPL_ENOMEM;
    if (rc == SPL_OK && cudaMallocHost((void **)&c->h_images, sizeof(float *) * kMaxViews) != cudaSuccess)
        rc = SPL_ENOMEM;
    if (rc == SPL_OK && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        rc = SPL_ECUDA;
    if (rc == SPL_OK) rc = c->heur.ensure(2);
    if (rc == SPL_OK) rc = c->theta.ensure(kNParam);
    if (rc == SPL_OK) rc = c->order_hist.ensure(512);
    if (rc == SPL_OK) {
        const float h0[2] = {0.f, 1.f};   // count heuristic: log1p(entries)
        if (cudaMemcpy(c->heur.p, h0, sizeof(h0), cudaMemcpyHostToDevice) != cudaSuccess) rc = SPL_ECUDA;
    }
    for (int k = 0; rc == SPL_OK && k < 12; ++k)
        if (cudaEventCreate(&c->ev[k / 6][k % 6]) != cudaSuccess) rc = SPL_ECUDA;
    if (rc == SPL_OK && cudaEventCreateWithFlags(&c->stats_ready, cudaEventDisableTiming) != cudaSuccess)
        rc = SPL_ECUDA;
    if (rc != SPL_OK) {
        cudaGetLastError();
        spl_destroy(c);
        return rc;
    }
    *out = c;
    return SPL_OK;
}

extern "C" int spl_destroy(spl_ctx *c) {
    if (!c) return SPL_OK;
    DeviceGuard g(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    c->x.release(); c->y.release(); c->z.release();
    c->h.release(); c->I.release(); c->s.release();
    c->cr.release(); c->cg.release(); c->cb.release();
    for (int b = 0; b < 2; ++b) {
        c->cx[b].release(); c->cy[b].release(); c->cz[b].release();
        c->ch[b].release(); c->cI[b].release(); c->cs[b].release();
        c->ccr[b].release(); c->ccg[b].release(); c->ccb[b].release();
        if (c->copied[b]) cudaEventDestroy(c->copied[b]);
        if (c->consumed[b]) cudaEventDestroy(c->consumed[b]);
    }
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    c->pal.release();
    c->recs.release();
    c->rec2.release(); c->pkeys.release(); c->ptmp.release(); c->ekeys.release();
    c->etmp.release(); c->rank.release(); c->sort_hist.release(); c->partial.release();
    c->counts.release(); c->offsets.release(); c->cursor.release();
    c->ovf.release(); c->ctab.release();
    c->large_ids.release(); c->entries.release(); c->dstats.release();
    c->item_counts.release(); c->item_offsets.release(); c->items.release();
    c->host_img_scratch.release();
    c->d_fcs.release(); c->d_images.release();
    c->feat.release(); c->cost.release(); c->theta.release(); c->heur.release();
    c->item_n.release(); c->order.release(); c->order_hist.release(); c->item_cycles.release();
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->hstats) cudaFreeHost(c->hstats);
    if (c->h_fcs) cudaFreeHost(c->h_fcs);
    if (c->h_images) cudaFreeHost(c->h_images);
    for (auto &set : c->ev)
        for (auto &e : set)
            if (e) cudaEventDestroy(e);
    if (c->stats_ready) cudaEventDestroy(c->stats_ready);
    delete c;
    return SPL_OK;
}

// Bytes per value of h and of I, s in a storage layout.
static size_t h_bytes(int attr) { return (attr == SPL_ATTR_F16 || attr == SPL_ATTR_LOGH16) ? 2 : 4; }
static size_t is_bytes(int attr) { return attr == SPL_ATTR_F32 ? 4 : 2; }

static bool particles_ok(const spl_particles *p) {
    if (!p || p->n < 0) return false;
    if (p->attr_type < SPL_ATTR_F32 || p->attr_type > SPL_ATTR_LOGH16) return false;
    if (p->attr_type == SPL_ATTR_LOGH16 && !std::isfinite(p->h_log2_min)) return false;
    if (p->mem_space != SPL_MEM_HOST && p->mem_space != SPL_MEM_DEVICE) return false;
    if (p->n > 0 && (!p->x || !p->y || !p->z || !p->h || !p->I || !p->s)) return false;
    const int nrgb = (p->cr != nullptr) + (p->cg != nullptr) + (p->cb != nullptr);
    if (nrgb != 0 && nrgb != 3) return false;
    return p->n <= (int64_t)0xFFFFFFFFLL;   // ids are 32-bit
}

// Copy a particle set into the context's SoA; the attributes are stored in
// layout `store` (p->attr_type, or any layout when p->attr_type is FP32: then
// the encoder converts them on the device).
static int load_impl(spl_ctx *c, const spl_particles *p, int store, float h_log2_min) {
    DeviceGuard g(c->device);
    const size_t n = (size_t)p->n;
    const size_t ah = h_bytes(store), ab = is_bytes(store);
    const bool convert = store != p->attr_type;
    SPL_TRY(c->x.ensure(n ? n : 1));
    SPL_TRY(c->y.ensure(n ? n : 1));
    SPL_TRY(c->z.ensure(n ? n : 1));
    SPL_TRY(c->h.ensure((n ? n : 1) * ah));
    SPL_TRY(c->I.ensure((n ? n : 1) * ab));
    SPL_TRY(c->s.ensure((n ? n : 1) * ab));
    const cudaMemcpyKind kind =
        p->mem_space == SPL_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    float *tmp = nullptr;   // device copies of host FP32 attributes to be converted
    if (convert && n && p->mem_space == SPL_MEM_HOST) {
        if (cudaMalloc((void **)&tmp, 3 * n * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            return SPL_ENOMEM;
        }
    }
    int rc = SPL_OK;
    auto copy = [&](void *dst, const void *src, size_t bytes) {
        if (rc == SPL_OK) rc = cuda_status(cudaMemcpyAsync(dst, src, bytes, kind, c->stream));
    };
    if (n) {
        copy(c->x.p, p->x, n * 4);
        copy(c->y.p, p->y, n * 4);
        copy(c->z.p, p->z, n * 4);
        if (!convert) {
            copy(c->h.p, p->h, n * ah);
            copy(c->I.p, p->I, n * ab);
            copy(c->s.p, p->s, n * ab);
        } else {
            const float *dh = static_cast<const float *>(p->h);
            const float *dI = static_cast<const float *>(p->I);
            const float *ds = static_cast<const float *>(p->s);
            if (tmp) {
                copy(tmp, p->h, n * 4);
                copy(tmp + n, p->I, n * 4);
                copy(tmp + 2 * n, p->s, n * 4);
                dh = tmp;
                dI = tmp + n;
                ds = tmp + 2 * n;
            }
            if (rc == SPL_OK) {
                launch_encode_attrs(dh, dI, ds, (int64_t)n, store, h_log2_min, c->h.p, c->I.p,
                                    c->s.p, c->sms, c->stream);
                rc = cuda_status(cudaGetLastError());
            }
        }
    }
    const bool rgb = p->cr != nullptr;
    if (rgb && rc == SPL_OK) {
        rc = c->cr.ensure(n ? n : 1);
        if (rc == SPL_OK) rc = c->cg.ensure(n ? n : 1);
        if (rc == SPL_OK) rc = c->cb.ensure(n ? n : 1);
        if (n) {
            copy(c->cr.p, p->cr, n * 4);
            copy(c->cg.p, p->cg, n * 4);
            copy(c->cb.p, p->cb, n * 4);
        }
    }
    if (rc == SPL_OK) rc = cuda_status(cudaStreamSynchronize(c->stream));
    if (tmp) cudaFree(tmp);
    if (rc != SPL_OK) return rc;
    c->have_rgb = rgb;
    c->n = p->n;
    c->attr_type = store;
    c->h_log2_min = store == SPL_ATTR_LOGH16 ? h_log2_min : 0.f;
    c->have_particles = true;
    return SPL_OK;
}

extern "C" int spl_load_particles(spl_ctx *c, const spl_particles *p) {
    if (!c || !particles_ok(p)) return SPL_EINVAL;
    return load_impl(c, p, p->attr_type, p->h_log2_min);
}

extern "C" int spl_load_particles_as(spl_ctx *c, const spl_particles *p, int32_t store_as,
                                     float h_log2_min) {
    if (!c || !particles_ok(p) || p->attr_type != SPL_ATTR_F32) return SPL_EINVAL;
    if (store_as < SPL_ATTR_F32 || store_as > SPL_ATTR_LOGH16) return SPL_EINVAL;
    if (store_as == SPL_ATTR_LOGH16 && !std::isfinite(h_log2_min)) return SPL_EINVAL;
    return load_impl(c, p, store_as, h_log2_min);
}

extern "C" int spl_encode_attrs(spl_ctx *c, const float *d_h, const float *d_I, const float *d_s,
                                int64_t n, int32_t store_as, float h_log2_min, void *d_h_out,
                                void *d_I_out, void *d_s_out, void *stream) {
    if (!c || n < 0) return SPL_EINVAL;
    if (store_as < SPL_ATTR_F32 || store_as > SPL_ATTR_LOGH16) return SPL_EINVAL;
    if (store_as == SPL_ATTR_LOGH16 && !std::isfinite(h_log2_min)) return SPL_EINVAL;
    if (n > 0 && (!d_h || !d_I || !d_s || !d_h_out || !d_I_out || !d_s_out)) return SPL_EINVAL;
    DeviceGuard g(c->device);
    launch_encode_attrs(d_h, d_I, d_s, n, store_as, h_log2_min, d_h_out, d_I_out, d_s_out, c->sms,
                        stream ? (cudaStream_t)stream : c->stream);
    return cuda_status(cudaGetLastError());
}

extern "C" int spl_apply_ea(spl_ctx *c, float *d_image, int64_t n_values, void *stream) {
    if (!c || n_values < 0 || (n_values > 0 && !d_image)) return SPL_EINVAL;
    DeviceGuard g(c->device);
    launch_epilogue_ea(d_image, n_values, c->sms, stream ? (cudaStream_t)stream : c->stream);
    return cuda_status(cudaGetLastError());
}

extern "C" int spl_set_camera(spl_ctx *c, const spl_camera *cam) {
    if (!c || !camera_ok(cam)) return SPL_EINVAL;
    c->cam = *cam;
    c->have_cam = true;
    return SPL_OK;
}

extern "C" int spl_set_colormap(spl_ctx *c, const float *rgb, int32_t n, float s_min, float s_max) {
    if (!c || !rgb || n < 1 || n > kMaxPalette) return SPL_EINVAL;
    if (!std::isfinite(s_min) || !std::isfinite(s_max)) return SPL_EINVAL;
    for (int k = 0; k < 3 * n; ++k)
        if (!std::isfinite(rgb[k])) return SPL_EINVAL;
    DeviceGuard g(c->device);
    SPL_TRY(c->pal.ensure((size_t)3 * n));
    SPL_CUDA(cudaMemcpyAsync(c->pal.p, rgb, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, c->stream));
    SPL_CUDA(cudaStreamSynchronize(c->stream));
    c->npal = n;
    c->s_min = s_min;
    c->s_max = s_max;
    return SPL_OK;
}

extern "C" int spl_set_params(spl_ctx *c, const spl_params *q) {
    if (!c || !params_ok(q)) return SPL_EINVAL;
    c->par = *q;
    return SPL_OK;
}

extern "C" int spl_get_params(spl_ctx *c, spl_params *out) {
    if (!c || !out) return SPL_EINVAL;
    *out = c->par;
    return SPL_OK;
}

extern "C" int spl_set_graph(spl_ctx *c, int32_t enable) {
    if (!c) return SPL_EINVAL;
    c->use_graph = enable != 0;
    return SPL_OK;
}

extern "C" int spl_set_timing(spl_ctx *c, int32_t enable) {
    if (!c) return SPL_EINVAL;
    c->timing = enable != 0;
    c->ev_pending[0] = c->ev_pending[1] = false;
    for (double &v : c->sum_ms) v = 0.0;
    c->timed_frames = 0;
    return SPL_OK;
}

// Read the stage times of event set k (its last event must have completed).
static void harvest_timing(spl_ctx *c, int k) {
    if (!c->ev_pending[k]) return;
    c->ev_pending[k] = false;
    for (int st = 0; st < 6; ++st) {
        const int a = st < 5 ? st : 0, b = st < 5 ? st + 1 : 5;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->ev[k][a], c->ev[k][b]) != cudaSuccess) {
            cudaGetLastError();
            ms = 0.f;
        }
        c->last_ms[st] = ms;
        c->sum_ms[st] += ms;
    }
    c->timed_frames += 1;
}

extern "C" int spl_get_stats(spl_ctx *c, spl_stats *out) {
    if (!c || !out) return SPL_EINVAL;
    DeviceGuard g(c->device);
    for (int q = 0; q < 2; ++q) {
        const int k = (c->ev_set + q) & 1;   // older set first
        if (c->ev_pending[k]) {
            SPL_CUDA(cudaEventSynchronize(c->ev[k][5]));
            harvest_timing(c, k);
        }
    }
    spl_stats &st = c->last;
    st.ms_raster = c->last_ms[0];
    st.ms_bin = c->last_ms[1];
    st.ms_tile = c->last_ms[2];
    st.ms_large = c->last_ms[3];
    st.ms_epilogue = c->last_ms[4];
    st.ms_total = c->last_ms[5];
    st.timed_frames = c->timed_frames;
    for (int k = 0; k < 6; ++k) st.sum_ms[k] = c->sum_ms[k];
    *out = st;
    return SPL_OK;
}

static void split_double(double v, float &hi, float &lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

// Per-frame constants: the look-at basis and focal length in double, handed
// to the device as double-float pairs.
static FrameConst make_frame(const spl_ctx *c, const spl_camera &cam) {
    FrameConst fc;
    std::memset(&fc, 0, sizeof(fc));
    double f[3], r[3], u[3];
    for (int k = 0; k < 3; ++k) f[k] = cam.target[k] - cam.eye[k];
    double nf = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    for (double &v : f) v /= nf;
    r[0] = f[1] * cam.up[2] - f[2] * cam.up[1];
    r[1] = f[2] * cam.up[0] - f[0] * cam.up[2];
    r[2] = f[0] * cam.up[1] - f[1] * cam.up[0];
    double nr = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    for (double &v : r) v /= nr;
    u[0] = r[1] * f[2] - r[2] * f[1];
    u[1] = r[2] * f[0] - r[0] * f[2];
    u[2] = r[0] * f[1] - r[1] * f[0];
    const double *rows[3] = {r, u, f};
    for (int a = 0; a < 3; ++a) {
        double e = 0;
        for (int b = 0; b < 3; ++b) {
            split_double(rows[a][b], fc.Rhi[3 * a + b], fc.Rlo[3 * a + b]);
            e += rows[a][b] * cam.eye[b];
        }
        split_double(e, fc.Ehi[a], fc.Elo[a]);
    }
    const double foc = 0.5 * cam.height / std::tan(0.5 * cam.fov_y_deg * M_PI / 180.0);
    split_double(foc, fc.fhi, fc.flo);
    fc.half_w = 0.5f * (float)cam.width;
    fc.half_h = 0.5f * (float)cam.height;
    fc.z_near = (float)cam.z_near;
    const spl_params &q = c->par;
    fc.sig_fac = (float)(q.sigma_per_h / q.s_box);
    fc.chi = (float)q.chi;
    fc.r_sml2 = (float)(q.r_sml * q.r_sml);
    fc.r_small2 = (float)(q.r_small * q.r_small);
    fc.r_large2 = (float)(q.r_large * q.r_large);
    fc.absorb = q.mode == SPL_MODE_ABSORB ? 1 : 0;
    fc.absorption = (float)q.absorption;
    fc.log_flags = q.log_flags;
    if (fc.absorb) {
        // one list per tile: no small class, no separate large pass
        fc.r_small2 = fc.r_sml2;
        fc.r_large2 = 3.0e38f;
    }
    fc.s_min = c->s_min;
    fc.s_inv = c->s_max != c->s_min ? (float)(1.0 / ((double)c->s_max - (double)c->s_min)) : 0.f;
    fc.brightness = (float)q.brightness;
    fc.npal = c->npal;
    fc.width = cam.width;
    fc.height = cam.height;
    fc.tile = q.tile_px;
    fc.tile_shift = q.tile_px == 16 ? 4 : (q.tile_px == 32 ? 5 : 6);
    fc.ntx = (cam.width + q.tile_px - 1) / q.tile_px;
    fc.nty = (cam.height + q.tile_px - 1) / q.tile_px;
    fc.ntiles = fc.ntx * fc.nty;
    return fc;
}

static void record_event(spl_ctx *c, int k, cudaStream_t s) {
    if (c->timing) cudaEventRecord(c->ev[c->ev_set][k], s);
}

// ---------------------------------------------------------------------------
// The pipeline over a batch of views (a single frame is a batch of one).
// ---------------------------------------------------------------------------

// Grow buffer b to n elements; note when it moved (a captured graph holds
// its old address).
template <typename T>
static int grow(spl_ctx *c, DevBuf<T> &b, size_t n) {
    if (n <= b.cap && b.p) return SPL_OK;
    c->buf_gen++;
    return b.ensure(n);
}

// Number of particles the pipeline reads: the loaded set, or the chunk being
// streamed.
static int64_t src_n(const spl_ctx *c) { return c->streaming ? c->chunk_n : c->n; }

// Per-view constants into the pinned staging; sizes every per-batch buffer
// that does not depend on the binning results.
static int prepare_views(spl_ctx *c, const spl_camera *cams, int V, float *const *images,
                         Views &vs) {
    if (V < 1 || V > kMaxViews) return SPL_EINVAL;
    int tiles = 0;
    for (int v = 0; v < V; ++v) {
        FrameConst fc = make_frame(c, cams[v]);
        fc.view = v;
        fc.tile_base = tiles;
        fc.slot_base = NLIST * tiles;
        fc.rec_base = (long long)v * src_n(c);
        if ((int64_t)tiles + fc.ntiles > (int64_t)0x7FFFFFFF / (2 * NLIST)) return SPL_EINVAL;
        tiles += fc.ntiles;
        c->h_fcs[v] = fc;
        c->h_images[v] = images[v];
    }
    if ((int64_t)V * src_n(c) > (int64_t)0xFFFFFFFFLL) return SPL_EINVAL;   // record ids are 32-bit
    const size_t recs = (size_t)V * (size_t)src_n(c);
    SPL_TRY(grow(c, c->recs, recs ? recs : 1));
    if (c->par.mode == SPL_MODE_ABSORB) {
        SPL_TRY(grow(c, c->rec2, recs ? recs : 1));
        SPL_TRY(grow(c, c->pkeys, recs ? recs : 1));
        SPL_TRY(grow(c, c->ptmp, recs ? recs : 1));
        SPL_TRY(grow(c, c->rank, recs ? recs : 1));
    }
    SPL_TRY(grow(c, c->large_ids, recs ? recs : 1));
    SPL_TRY(grow(c, c->counts, (size_t)NLIST * tiles));
    SPL_TRY(grow(c, c->ovf, (size_t)NLIST * tiles));
    SPL_TRY(grow(c, c->ctab, (size_t)ctab_entries(src_n(c), V)));
    SPL_TRY(grow(c, c->offsets, (size_t)NLIST * tiles + 1));
    SPL_TRY(grow(c, c->cursor, (size_t)NLIST * tiles));
    SPL_TRY(grow(c, c->item_counts, (size_t)2 * tiles));
    SPL_TRY(grow(c, c->item_offsets, (size_t)2 * tiles + 1));
    SPL_TRY(grow(c, c->entries, 16));
    SPL_TRY(grow(c, c->items, 16));
    SPL_TRY(grow(c, c->d_fcs, kMaxViews));
    SPL_TRY(grow(c, c->d_images, kMaxViews));
    vs.fcs = c->d_fcs.p;
    vs.nviews = V;
    vs.total_tiles = tiles;
    vs.tile = c->par.tile_px;
    vs.n = src_n(c);
    return SPL_OK;
}

// Per-item buffers follow the capacity of the item array.
static int size_item_buffers(spl_ctx *c) {
    const size_t n = c->items.cap;
    SPL_TRY(grow(c, c->feat, n * kFeat));
    SPL_TRY(grow(c, c->cost, n));
    SPL_TRY(grow(c, c->item_n, n));
    SPL_TRY(grow(c, c->order, n));
    SPL_TRY(grow(c, c->item_cycles, n));
    return SPL_OK;
}

// Stage 1: constants to the device, rasterise every view, count and scan the
// list slots and the work items.
static void enqueue_binning(spl_ctx *c, const Views &vs, cudaStream_t s) {
    cudaMemcpyAsync(c->d_fcs.p, c->h_fcs, sizeof(FrameConst) * vs.nviews, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(c->d_images.p, c->h_images, sizeof(float *) * vs.nviews, cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(c->counts.p, 0, sizeof(int) * NLIST * vs.total_tiles, s);
    cudaMemsetAsync(c->ovf.p, 0, sizeof(int) * NLIST * vs.total_tiles, s);
    cudaMemsetAsync(c->dstats.p, 0, offsetof(DevStats, err), s);
    RasterArgs ra{};
    ra.n = src_n(c);
    if (c->streaming) {
        const int b = c->chunk_buf;
        ra.x = c->cx[b].p; ra.y = c->cy[b].p; ra.z = c->cz[b].p;
        ra.h = c->ch[b].p; ra.I = c->cI[b].p; ra.s = c->cs[b].p;
        if (c->chunk_rgb) {
            ra.cr = c->ccr[b].p; ra.cg = c->ccg[b].p; ra.cb = c->ccb[b].p;
        }
        ra.h_log2_min = c->chunk_h_log2_min;
    } else {
        ra.x = c->x.p; ra.y = c->y.p; ra.z = c->z.p;
        ra.h = c->h.p; ra.I = c->I.p; ra.s = c->s.p;
        if (c->have_rgb) {
            ra.cr = c->cr.p; ra.cg = c->cg.p; ra.cb = c->cb.p;
        }
        ra.h_log2_min = c->h_log2_min;
    }
    ra.pal = c->pal.p;
    ra.recs = c->recs.p;
    ra.rec2 = c->par.mode == SPL_MODE_ABSORB ? c->rec2.p : nullptr;
    ra.counts = c->counts.p;
    ra.ovf = c->ovf.p;
    ra.ctab = c->ctab.p;
    ra.large_ids = c->large_ids.p;
    ra.st = c->dstats.p;
    launch_raster(vs, ra, c->streaming ? c->chunk_attr : c->attr_type, s);
    record_event(c, 1, s);
    BinArgs ba{};
    ba.recs = c->recs.p;
    ba.large_ids = c->large_ids.p;
    ba.counts = c->counts.p;
    ba.ovf = c->ovf.p;
    ba.cursor = c->cursor.p;
    ba.st = c->dstats.p;
    launch_count_large(vs, ba, c->sms, s);
    launch_slot_offsets(NLIST * vs.total_tiles, c->counts.p, c->ovf.p, c->offsets.p, c->cursor.p,
                        &c->dstats.p->slot_total, s);
    launch_item_counts(vs, c->offsets.p, c->item_counts.p, c->dstats.p, s);
    launch_scan(2 * vs.total_tiles, c->item_counts.p, c->item_offsets.p, nullptr, 2,
                c->dstats.p->item_totals, s);
}

// Stage 2: clear the images and fill the tile lists and work items into the
// current capacities (the kernels check them and flag an overflow instead of
// writing past the end).
static void enqueue_lists(spl_ctx *c, const Views &vs, cudaStream_t s) {
    if (!c->accumulate) launch_zero_images(vs, c->d_images.p, c->sms, s);
    BinArgs ba{};
    ba.recs = c->recs.p;
    ba.large_ids = c->large_ids.p;
    ba.counts = c->counts.p;
    ba.ovf = c->ovf.p;
    ba.offsets = c->offsets.p;
    ba.ctab = c->ctab.p;
    ba.cursor = c->cursor.p;
    ba.entries = c->entries.p;
    ba.entries_cap = (int64_t)c->entries.cap;
    ba.st = c->dstats.p;
    launch_scatter(vs, ba, c->sms, s);
    launch_fill_items(vs, c->offsets.p, c->item_offsets.p, c->items.p, (int)c->items.cap,
                      c->dstats.p, s);
}

// Stage 3: schedule the work items, the tile and large passes, the epilogue.
static void enqueue_passes(spl_ctx *c, const Views &vs, bool large_pass, cudaStream_t s) {
    TileArgs ta{};
    ta.recs = c->recs.p;
    ta.offsets = c->offsets.p;
    ta.entries = c->entries.p;
    ta.items = c->items.p;
    ta.items_cap = (int)c->items.cap;
    ta.images = c->d_images.p;
    ta.st = c->dstats.p;
    ta.accumulate = c->accumulate ? 1 : 0;
    // scheduling: per-item features, predicted cost, longest first
    const bool sched = c->par.sched != SPL_SCHED_NONE;
    const float *theta = c->par.sched == SPL_SCHED_MLP && c->have_model ? c->theta.p : nullptr;
    // exact features when recording training samples, else a 64-entry sample;
    // the count heuristic needs only the entry counts
    if (c->recording || theta)
        launch_item_features(vs, ta, (float)vs.tile * (float)vs.tile, c->recording ? 0 : 64,
                             c->feat.p, c->item_n.p, c->sms, s);
    else if (sched)
        launch_item_entries(vs, ta, c->item_n.p, c->sms, s);
    if (sched) {
        launch_item_cost(c->feat.p, c->item_n.p, theta, c->heur.p, ta.items_cap, c->dstats.p,
                         c->cost.p, s);
        launch_order_items(c->cost.p, ta.items_cap, c->dstats.p, c->order_hist.p, c->order.p, s);
        ta.order = c->order.p;
    }
    if (c->recording) ta.item_cycles = c->item_cycles.p;
    if (c->par.mode == SPL_MODE_ABSORB) {
        // one view: every entry sits in the medium slots [L_MEDIUM * nt, (L_MEDIUM + 1) * nt]
        const int nt = c->h_fcs[0].ntiles;
        launch_depth_order(c->recs.p, c->rec2.p, vs.n, c->entries.p, c->offsets.p + L_MEDIUM * nt,
                           nt, (long long)c->hstats->slot_total, c->pkeys.p, c->ptmp.p,
                           c->ekeys.p, c->etmp.p, c->rank.p, c->sort_hist.p, c->sms, s);
        ta.rec2 = c->rec2.p;
        ta.partial = c->partial.p;
        record_event(c, 2, s);
        launch_absorb_pass(vs, ta, c->item_offsets.p, c->sms, s);
        record_event(c, 3, s);
        record_event(c, 4, s);
        record_event(c, 5, s);
        return;
    }
    record_event(c, 2, s);
    launch_tile_pass(vs, ta, c->sms, s);
    record_event(c, 3, s);
    if (large_pass) launch_large_pass(vs, ta, c->sms, s);
    record_event(c, 4, s);
    if (c->par.mode == SPL_MODE_EA && c->last_chunk) launch_epilogue_views(vs, c->d_images.p, c->sms, s);
    record_event(c, 5, s);
}

static void fill_stats(spl_ctx *c, const Views &vs, int launches) {
    spl_stats &st = c->last;
    std::memset(&st, 0, sizeof(st));
    st.launches = launches;
    st.n_particles = src_n(c);
    st.n_active = (int64_t)c->hstats->n_active;
    st.n_point = (int64_t)c->hstats->n_point;
    st.n_small = (int64_t)c->hstats->n_small;
    st.n_medium = (int64_t)c->hstats->n_medium;
    st.n_large = (int64_t)c->hstats->n_large;
    for (int k = 0; k < NLIST; ++k) st.n_entries[k] = c->hstats->totals[k];
    st.n_tiles = vs.total_tiles;
    st.tile_px = vs.tile;
}

// Eager render of a batch.  The binning counts are copied to the host and the
// host waits for them (not for the stream): meanwhile the device clears the
// images and fills the tile lists into the capacities of the earlier frames.
// If the counts show that the lists or the work items did not fit, the host
// waits for that fill, grows the buffers, re-arms the list cursors and fills
// the lists again; either way the passes follow.
static int render_views(spl_ctx *c, const spl_camera *cams, int V, float *const *images,
                        cudaStream_t s) {
    if ((!c->have_particles && !c->streaming) || c->npal < 1) return SPL_ESTATE;
    Views vs{};
    SPL_TRY(prepare_views(c, cams, V, images, vs));
    SPL_CUDA(cudaGetLastError());
    const long long launched0 = g_launches;
    record_event(c, 0, s);
    enqueue_binning(c, vs, s);
    SPL_CUDA(cudaGetLastError());
    SPL_CUDA(cudaMemcpyAsync(c->hstats, c->dstats.p, sizeof(DevStats), cudaMemcpyDeviceToHost, s));
    SPL_CUDA(cudaEventRecord(c->stats_ready, s));
    enqueue_lists(c, vs, s);
    SPL_CUDA(cudaGetLastError());
    SPL_CUDA(cudaEventSynchronize(c->stats_ready));
    harvest_timing(c, c->ev_set ^ 1);   // the previous frame has finished
    if (c->hstats->err) {
        // a device-side check failed in an earlier frame: report it (the flag
        // is cleared once the lists queued above are done)
        SPL_CUDA(cudaStreamSynchronize(s));
        SPL_CUDA(cudaMemsetAsync(&c->dstats.p->err, 0, sizeof(unsigned), s));
        return SPL_EDEVICE;
    }
    const int64_t total = c->hstats->slot_total;
    const int n_tile_items = c->hstats->item_totals[0];
    const int n_large_items = c->hstats->item_totals[1];
    if ((size_t)total > c->entries.cap || (size_t)n_tile_items + n_large_items > c->items.cap) {
        // the lists ran into buffers too small: wait for them, grow, refill
        SPL_CUDA(cudaStreamSynchronize(s));
        SPL_TRY(grow(c, c->entries, (size_t)(total ? total : 1)));
        SPL_TRY(grow(c, c->items, (size_t)(n_tile_items + n_large_items + 1)));
        SPL_CUDA(cudaMemsetAsync(&c->dstats.p->err, 0, sizeof(unsigned), s));
        launch_slot_cursor(NLIST * vs.total_tiles, c->counts.p, c->offsets.p, c->cursor.p, s);
        enqueue_lists(c, vs, s);
        SPL_CUDA(cudaGetLastError());
    }
    SPL_TRY(size_item_buffers(c));
    if (c->par.mode == SPL_MODE_ABSORB) {
        const int64_t m = total > vs.n ? total : vs.n;
        SPL_TRY(grow(c, c->ekeys, (size_t)(total ? total : 1)));
        SPL_TRY(grow(c, c->etmp, (size_t)(total ? total : 1)));
        SPL_TRY(grow(c, c->sort_hist, (size_t)radix_scratch_ints(m)));
        SPL_TRY(grow(c, c->partial, c->items.cap * (size_t)vs.tile * (size_t)vs.tile));
    }
    c->last_items = n_tile_items + n_large_items;
    enqueue_passes(c, vs, n_large_items > 0, s);
    SPL_CUDA(cudaGetLastError());
    const int launches = (int)(g_launches - launched0);
    if (c->timing) {
        c->ev_pending[c->ev_set] = true;
        c->ev_set ^= 1;
    }
    fill_stats(c, vs, launches);
    return SPL_OK;
}

extern "C" int spl_render(spl_ctx *c, float *d_image, void *stream) {
    if (!c || !d_image) return SPL_EINVAL;
    if (!c->have_cam) return SPL_ESTATE;
    DeviceGuard g(c->device);
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    return render_views(c, &c->cam, 1, &d_image, s);
}

extern "C" int spl_render_host(spl_ctx *c, float *h_image) {
    if (!c || !h_image) return SPL_EINVAL;
    if (!c->have_cam) return SPL_ESTATE;
    DeviceGuard g(c->device);
    const size_t nv = (size_t)3 * c->cam.width * c->cam.height;
    SPL_TRY(c->host_img_scratch.ensure(nv));
    float *img = c->host_img_scratch.p;
    SPL_TRY(render_views(c, &c->cam, 1, &img, c->stream));
    SPL_CUDA(cudaMemcpyAsync(h_image, c->host_img_scratch.p, nv * sizeof(float),
                             cudaMemcpyDeviceToHost, c->stream));
    SPL_CUDA(cudaStreamSynchronize(c->stream));
    return SPL_OK;
}

// Configuration a captured batch graph is valid for: everything that shapes
// the launches or the buffer sizes (cameras themselves may change: their
// constants are copied from the pinned staging at replay time).
// Out-of-core render (Sec. 3.2, Eq. 3): the particles stay in host memory
// and pass through the device in chunks; chunk k+1 is copied on the copy
// stream while chunk k's tile lists are filled and rendered on the render
// stream (two device buffers, events in both directions), and every chunk
// adds its additive image into d_image (the sum is linear in the particle
// set, Sec. 2); the E=A map, if selected, follows the last chunk.
static int copy_chunk(spl_ctx *c, const spl_particles *p, int64_t first, int64_t cnt, int b) {
    const size_t ah = (p->attr_type == SPL_ATTR_F16 || p->attr_type == SPL_ATTR_LOGH16) ? 2 : 4;
    const size_t ab = p->attr_type == SPL_ATTR_F32 ? 4 : 2;
    const size_t m = (size_t)cnt;
    cudaStream_t cs = c->copy_stream;
    SPL_CUDA(cudaStreamWaitEvent(cs, c->consumed[b], 0));
    SPL_CUDA(cudaMemcpyAsync(c->cx[b].p, p->x + first, m * 4, cudaMemcpyHostToDevice, cs));
    SPL_CUDA(cudaMemcpyAsync(c->cy[b].p, p->y + first, m * 4, cudaMemcpyHostToDevice, cs));
    SPL_CUDA(cudaMemcpyAsync(c->cz[b].p, p->z + first, m * 4, cudaMemcpyHostToDevice, cs));
    SPL_CUDA(cudaMemcpyAsync(c->ch[b].p, (const unsigned char *)p->h + first * ah, m * ah,
                             cudaMemcpyHostToDevice, cs));
    SPL_CUDA(cudaMemcpyAsync(c->cI[b].p, (const unsigned char *)p->I + first * ab, m * ab,
                             cudaMemcpyHostToDevice, cs));
    SPL_CUDA(cudaMemcpyAsync(c->cs[b].p, (const unsigned char *)p->s + first * ab, m * ab,
                             cudaMemcpyHostToDevice, cs));
    if (p->cr) {
        SPL_CUDA(cudaMemcpyAsync(c->ccr[b].p, p->cr + first, m * 4, cudaMemcpyHostToDevice, cs));
        SPL_CUDA(cudaMemcpyAsync(c->ccg[b].p, p->cg + first, m * 4, cudaMemcpyHostToDevice, cs));
        SPL_CUDA(cudaMemcpyAsync(c->ccb[b].p, p->cb + first, m * 4, cudaMemcpyHostToDevice, cs));
    }
    SPL_CUDA(cudaEventRecord(c->copied[b], cs));
    return SPL_OK;
}

extern "C" int spl_render_stream(spl_ctx *c, const spl_particles *p, int64_t chunk, float *d_image,
                                 void *stream) {
    if (!c || !p || !d_image || chunk < 1 || p->n < 0) return SPL_EINVAL;
    if (p->attr_type < SPL_ATTR_F32 || p->attr_type > SPL_ATTR_LOGH16) return SPL_EINVAL;
    if (p->attr_type == SPL_ATTR_LOGH16 && !std::isfinite(p->h_log2_min)) return SPL_EINVAL;
    if (p->mem_space != SPL_MEM_HOST) return SPL_EINVAL;
    if (p->n > 0 && (!p->x || !p->y || !p->z || !p->h || !p->I || !p->s)) return SPL_EINVAL;
    const int nrgb = (p->cr != nullptr) + (p->cg != nullptr) + (p->cb != nullptr);
    if (nrgb != 0 && nrgb != 3) return SPL_EINVAL;
    if (!c->have_cam) return SPL_ESTATE;
    if (c->npal < 1) return SPL_ESTATE;
    if (c->par.mode == SPL_MODE_ABSORB) return SPL_EINVAL;   // not additive over chunks
    DeviceGuard g(c->device);
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    if (!c->copy_stream) {
        SPL_CUDA(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
        for (int b = 0; b < 2; ++b) {
            SPL_CUDA(cudaEventCreateWithFlags(&c->copied[b], cudaEventDisableTiming));
            SPL_CUDA(cudaEventCreateWithFlags(&c->consumed[b], cudaEventDisableTiming));
        }
    }
    const int64_t per = p->n < chunk ? (p->n > 0 ? p->n : 1) : chunk;
    const size_t ah = (p->attr_type == SPL_ATTR_F16 || p->attr_type == SPL_ATTR_LOGH16) ? 2 : 4;
    const size_t ab = p->attr_type == SPL_ATTR_F32 ? 4 : 2;
    for (int b = 0; b < 2; ++b) {
        SPL_TRY(c->cx[b].ensure((size_t)per));
        SPL_TRY(c->cy[b].ensure((size_t)per));
        SPL_TRY(c->cz[b].ensure((size_t)per));
        SPL_TRY(c->ch[b].ensure((size_t)per * ah));
        SPL_TRY(c->cI[b].ensure((size_t)per * ab));
        SPL_TRY(c->cs[b].ensure((size_t)per * ab));
        if (nrgb == 3) {
            SPL_TRY(c->ccr[b].ensure((size_t)per));
            SPL_TRY(c->ccg[b].ensure((size_t)per));
            SPL_TRY(c->ccb[b].ensure((size_t)per));
        }
        SPL_CUDA(cudaEventRecord(c->consumed[b], s));   // the buffers are free from here on
    }
    const int64_t nchunks = p->n > 0 ? (p->n + chunk - 1) / chunk : 1;
    int64_t tot[5] = {}, ents[4] = {};
    int rc = SPL_OK;
    if (p->n > 0) rc = copy_chunk(c, p, 0, per < p->n ? per : p->n, 0);
    c->streaming = true;
    c->chunk_attr = p->attr_type;
    c->chunk_h_log2_min = p->h_log2_min;
    c->chunk_rgb = nrgb == 3;
    for (int64_t k = 0; k < nchunks && rc == SPL_OK; ++k) {
        const int b = (int)(k & 1);
        const int64_t first = k * chunk;
        const int64_t cnt = p->n > 0 ? (p->n - first < chunk ? p->n - first : chunk) : 0;
        if (cnt > 0) {
            rc = cuda_status(cudaStreamWaitEvent(s, c->copied[b], 0));
            if (rc != SPL_OK) break;
        }
        c->chunk_buf = b;
        c->chunk_n = cnt;
        c->accumulate = k > 0;
        c->last_chunk = k + 1 == nchunks;
        rc = render_views(c, &c->cam, 1, &d_image, s);
        if (rc != SPL_OK) break;
        rc = cuda_status(cudaEventRecord(c->consumed[b], s));
        // the next chunk's copy starts once this chunk's binning is done (render_views
        // has synchronised after it), so that it overlaps the scatter and tile pass
        // and does not queue the small per-chunk uploads behind a large copy
        if (rc == SPL_OK && k + 1 < nchunks) {
            const int64_t nf = first + chunk;
            rc = copy_chunk(c, p, nf, p->n - nf < chunk ? p->n - nf : chunk, b ^ 1);
        }
        const spl_stats &st = c->last;
        tot[0] += st.n_active; tot[1] += st.n_point; tot[2] += st.n_small;
        tot[3] += st.n_medium; tot[4] += st.n_large;
        for (int l = 0; l < 4; ++l) ents[l] += st.n_entries[l];
    }
    c->streaming = false;
    c->accumulate = false;
    c->last_chunk = true;
    // the copy stream must not outlive the caller's host buffers
    const int rc2 = cuda_status(cudaStreamSynchronize(c->copy_stream));
    if (rc != SPL_OK) return rc;
    c->last.n_particles = p->n;
    c->last.n_active = tot[0];
    c->last.n_point = tot[1];
    c->last.n_small = tot[2];
    c->last.n_medium = tot[3];
    c->last.n_large = tot[4];
    for (int l = 0; l < 4; ++l) c->last.n_entries[l] = ents[l];
    return rc2;
}

static unsigned long long batch_key(const spl_ctx *c, const spl_camera *cams, int V) {
    unsigned long long h = 1469598103934665603ULL;
    auto mix = [&h](const void *p, size_t n) {
        const unsigned char *b = static_cast<const unsigned char *>(p);
        for (size_t k = 0; k < n; ++k) h = (h ^ b[k]) * 1099511628211ULL;
    };
    mix(&V, sizeof(V));
    for (int v = 0; v < V; ++v) {
        mix(&cams[v].width, sizeof(cams[v].width));
        mix(&cams[v].height, sizeof(cams[v].height));
    }
    mix(&c->par, sizeof(c->par));
    mix(&c->n, sizeof(c->n));
    mix(&c->attr_type, sizeof(c->attr_type));
    mix(&c->have_rgb, sizeof(c->have_rgb));
    mix(&c->h_log2_min, sizeof(c->h_log2_min));
    mix(&c->npal, sizeof(c->npal));
    mix(&c->buf_gen, sizeof(c->buf_gen));
    return h;
}

// Capture the whole batch pipeline (no host synchronisation inside) on the
// private capture stream; list and item capacities are the current ones.
static int capture_batch(spl_ctx *c, const Views &vs, unsigned long long key) {
    if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    const bool timing = c->timing;
    c->timing = false;   // no events inside the graph
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        const long long launched0 = g_launches;
        enqueue_binning(c, vs, c->cap_stream);
        enqueue_lists(c, vs, c->cap_stream);
        enqueue_passes(c, vs, true, c->cap_stream);
        c->graph_kernels = (int)(g_launches - launched0);
        e = cudaStreamEndCapture(c->cap_stream, &g);
    }
    c->timing = timing;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->graph = nullptr;
        return SPL_ECUDA;
    }
    c->graph_key = key;
    return SPL_OK;
}

extern "C" int spl_render_batch(spl_ctx *c, const spl_camera *cams, int32_t n_views,
                                float *const *d_images, void *stream) {
    if (!c || !cams || !d_images || n_views < 0 || n_views > kMaxViews) return SPL_EINVAL;
    for (int v = 0; v < n_views; ++v)
        if (!camera_ok(&cams[v]) || !d_images[v]) return SPL_EINVAL;
    if (n_views == 0) return SPL_OK;
    if (!c->have_particles || c->npal < 1) return SPL_ESTATE;
    if (c->par.mode == SPL_MODE_ABSORB) return SPL_EINVAL;   // single views only
    DeviceGuard g(c->device);
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    const unsigned long long key = batch_key(c, cams, n_views);
    if (c->use_graph && c->graph && c->graph_key == key) {
        // replay: stage the constants, launch, check the device-side guards
        Views vs{};
        SPL_TRY(prepare_views(c, cams, n_views, d_images, vs));
        if (batch_key(c, cams, n_views) == key) {
            record_event(c, 0, s);
            SPL_CUDA(cudaGraphLaunch(c->graph, s));
            record_event(c, 5, s);
            SPL_CUDA(cudaMemcpyAsync(c->hstats, c->dstats.p, sizeof(DevStats),
                                     cudaMemcpyDeviceToHost, s));
            SPL_CUDA(cudaStreamSynchronize(s));
            if (!c->hstats->err) {
                if (c->timing) {
                    // only the total is timed inside a graph
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, c->ev[c->ev_set][0], c->ev[c->ev_set][5]);
                    for (int k = 0; k < 6; ++k) c->last_ms[k] = 0.f;
                    c->last_ms[5] = ms;
                    c->sum_ms[5] += ms;
                    c->timed_frames += 1;
                }
                fill_stats(c, vs, c->graph_kernels);
                return SPL_OK;
            }
            // a list outgrew its captured capacity: clear and render eagerly
            SPL_CUDA(cudaMemsetAsync(&c->dstats.p->err, 0, sizeof(unsigned), s));
            SPL_CUDA(cudaStreamSynchronize(s));
        }
    }
    // eager render (exact list sizes), then capture a graph for the next call
    SPL_TRY(render_views(c, cams, n_views, d_images, s));
    if (!c->use_graph) return SPL_OK;
    SPL_CUDA(cudaStreamSynchronize(s));
    harvest_timing(c, c->ev_set ^ 1);
    Views vs{};
    SPL_TRY(prepare_views(c, cams, n_views, d_images, vs));
    // headroom so that small changes of the cameras still fit the graph: a
    // quarter above what the eager render needed (not above the capacity, which
    // would compound over re-captures)
    const size_t need_e = (size_t)(c->hstats->slot_total > 0 ? c->hstats->slot_total : 1);
    const size_t need_i = (size_t)c->last_items + 1;
    SPL_TRY(grow(c, c->entries, need_e + need_e / 4));
    SPL_TRY(grow(c, c->items, need_i + need_i / 4));
    SPL_TRY(size_item_buffers(c));
    SPL_TRY(capture_batch(c, vs, batch_key(c, cams, n_views)));
    return SPL_OK;
}

// ---------------------------------------------------------------------------
// Autotuner: tile side and class radii for a batch (Sec. 5.1 tunes n_p and
// t_x empirically for occupancy; here the candidates are timed directly).
// ---------------------------------------------------------------------------
extern "C" int spl_autotune(spl_ctx *c, const spl_camera *cams, int32_t n_views,
                            float *const *d_images, int32_t reps, spl_params *best,
                            float *best_ms) {
    if (!c || !cams || !d_images || n_views < 1 || n_views > kMaxViews || reps < 1) return SPL_EINVAL;
    for (int v = 0; v < n_views; ++v)
        if (!camera_ok(&cams[v]) || !d_images[v]) return SPL_EINVAL;
    if (!c->have_particles || c->npal < 1) return SPL_ESTATE;
    if (c->par.mode == SPL_MODE_ABSORB) return SPL_EINVAL;   // single views only
    DeviceGuard g(c->device);
    static const int tiles[] = {16, 32, 64};
    static const double radii[][2] = {{2.0, 32.0}, {2.0, 64.0}, {2.0, 128.0}, {2.0, 1e9}, {3.0, 64.0}, {0.0, 64.0}};
    const spl_params base = c->par;
    spl_params bp = base;
    float bms = -1.f;
    cudaStream_t s = c->stream;
    const bool timing = c->timing;
    c->timing = false;
    cudaEvent_t e0 = c->ev[0][0], e1 = c->ev[0][5];
    int rc = SPL_OK;
    for (int t : tiles) {
        for (const auto &rr : radii) {
            spl_params q = base;
            q.tile_px = t;
            q.r_small = rr[0] > q.r_sml ? rr[0] : q.r_sml;
            q.r_large = rr[1] > q.r_small ? rr[1] : q.r_small;
            if (!params_ok(&q)) continue;
            c->par = q;
            rc = render_views(c, cams, n_views, d_images, s);   // warm-up, sizes the lists
            if (rc != SPL_OK) break;
            cudaEventRecord(e0, s);
            for (int k = 0; k < reps && rc == SPL_OK; ++k) rc = render_views(c, cams, n_views, d_images, s);
            cudaEventRecord(e1, s);
            if (rc != SPL_OK) break;
            rc = cuda_status(cudaEventSynchronize(e1));
            if (rc != SPL_OK) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= reps;
            if (bms < 0.f || ms < bms) {
                bms = ms;
                bp = q;
            }
        }
        if (rc != SPL_OK) break;
    }
    c->timing = timing;
    c->ev_pending[0] = c->ev_pending[1] = false;
    c->par = rc == SPL_OK ? bp : base;
    if (rc != SPL_OK) return rc;
    if (best) *best = bp;
    if (best_ms) *best_ms = bms;
    return SPL_OK;
}

// ---------------------------------------------------------------------------
// Tile-cost network: model, samples, kernels, training.
// ---------------------------------------------------------------------------
extern "C" int spl_set_model(spl_ctx *c, const float *theta, const float *heur) {
    if (!c) return SPL_EINVAL;
    DeviceGuard g(c->device);
    if (theta) {
        for (int k = 0; k < kNParam; ++k)
            if (!std::isfinite(theta[k])) return SPL_EINVAL;
        SPL_CUDA(cudaMemcpy(c->theta.p, theta, sizeof(float) * kNParam, cudaMemcpyHostToDevice));
        c->have_model = true;
    }
    if (heur) {
        if (!std::isfinite(heur[0]) || !std::isfinite(heur[1])) return SPL_EINVAL;
        SPL_CUDA(cudaMemcpy(c->heur.p, heur, sizeof(float) * 2, cudaMemcpyHostToDevice));
    }
    return SPL_OK;
}

extern "C" int spl_set_recording(spl_ctx *c, int32_t enable) {
    if (!c) return SPL_EINVAL;
    c->recording = enable != 0;
    return SPL_OK;
}

extern "C" int spl_get_samples(spl_ctx *c, float *d_feat, float *d_logc, int64_t cap, int64_t *n) {
    if (!c || !n || cap < 0 || (cap > 0 && (!d_feat || !d_logc))) return SPL_EINVAL;
    if (!c->recording) return SPL_ESTATE;
    DeviceGuard g(c->device);
    SPL_CUDA(cudaStreamSynchronize(c->stream));
    const int64_t m = c->last_items < cap ? c->last_items : cap;
    if (m > 0) {
        SPL_CUDA(cudaMemcpy(d_feat, c->feat.p, sizeof(float) * kFeat * m, cudaMemcpyDeviceToDevice));
        launch_log_cycles(c->item_cycles.p, m, d_logc, c->stream);
        SPL_CUDA(cudaGetLastError());
        SPL_CUDA(cudaStreamSynchronize(c->stream));
    }
    *n = m;
    return SPL_OK;
}

extern "C" int spl_mlp_nparam(void) { return kNParam; }

extern "C" int spl_mlp_forward(const float *d_theta, const float *d_x, int64_t B, float *d_y,
                               void *stream) {
    if (!d_theta || B < 0 || (B > 0 && (!d_x || !d_y))) return SPL_EINVAL;
    launch_mlp_forward(d_theta, d_x, B, d_y, (cudaStream_t)stream);
    return cuda_status(cudaGetLastError());
}

extern "C" int spl_mlp_loss_grad(const float *d_theta, const float *d_x, const float *d_t, int64_t B,
                                 float *d_grad, float *d_loss, void *stream) {
    if (!d_theta || !d_grad || B < 1 || !d_x || !d_t) return SPL_EINVAL;
    float *work = nullptr;
    if (cudaMalloc((void **)&work, sizeof(float) * mlp_work_floats(B)) != cudaSuccess) {
        cudaGetLastError();
        return SPL_ENOMEM;
    }
    cudaStream_t s = (cudaStream_t)stream;
    launch_mlp_loss_grad(d_theta, d_x, d_t, B, work, d_grad, d_loss, s);
    int rc = cuda_status(cudaGetLastError());
    if (rc == SPL_OK) rc = cuda_status(cudaStreamSynchronize(s));
    cudaFree(work);
    return rc;
}

extern "C" int spl_mlp_adam(float *d_theta, const float *d_grad, float *d_m, float *d_v, int64_t np,
                            int64_t step, float lr, float beta1, float beta2, float eps,
                            void *stream) {
    if (!d_theta || !d_grad || !d_m || !d_v || np < 0 || step < 1) return SPL_EINVAL;
    launch_mlp_adam(d_theta, d_grad, d_m, d_v, np, step, lr, beta1, beta2, eps, (cudaStream_t)stream);
    return cuda_status(cudaGetLastError());
}

extern "C" int spl_mlp_train(const float *d_x, const float *d_t, int64_t B, float *theta,
                             int32_t steps, float lr, float *losses, void *stream) {
    if (!d_x || !d_t || B < 1 || !theta || steps < 0 || !(lr > 0.f)) return SPL_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    float *buf = nullptr;
    const size_t nf = 4 * (size_t)kNParam + (size_t)(steps + 1) + mlp_work_floats(B);
    if (cudaMalloc((void **)&buf, sizeof(float) * nf) != cudaSuccess) {
        cudaGetLastError();
        return SPL_ENOMEM;
    }
    float *th = buf, *gr = th + kNParam, *m = gr + kNParam, *v = m + kNParam;
    float *ls = v + kNParam, *work = ls + steps + 1;
    int rc = cuda_status(cudaMemcpyAsync(th, theta, sizeof(float) * kNParam, cudaMemcpyHostToDevice, s));
    if (rc == SPL_OK) rc = cuda_status(cudaMemsetAsync(m, 0, sizeof(float) * 2 * kNParam, s));
    for (int k = 0; rc == SPL_OK && k < steps; ++k) {
        launch_mlp_loss_grad(th, d_x, d_t, B, work, gr, ls + k, s);
        launch_mlp_adam(th, gr, m, v, kNParam, k + 1, lr, 0.9f, 0.999f, 1e-8f, s);
    }
    if (rc == SPL_OK) rc = cuda_status(cudaGetLastError());
    if (rc == SPL_OK) rc = cuda_status(cudaMemcpyAsync(theta, th, sizeof(float) * kNParam,
                                                       cudaMemcpyDeviceToHost, s));
    if (rc == SPL_OK && losses && steps > 0)
        rc = cuda_status(cudaMemcpyAsync(losses, ls, sizeof(float) * steps, cudaMemcpyDeviceToHost, s));
    if (rc == SPL_OK) rc = cuda_status(cudaStreamSynchronize(s));
    cudaFree(buf);
    return rc;
}

extern "C" int spl_get_records(spl_ctx *c, int64_t n, double *xs, double *ys, float *r, float *e,
                               int32_t *cls) {
    if (!c || n < 0 || n > c->n) return SPL_EINVAL;
    if (n == 0) return SPL_OK;
    if ((size_t)n > c->recs.cap) return SPL_ESTATE;
    DeviceGuard g(c->device);
    float4 *h0 = new (std::nothrow) float4[n];
    float4 *h1 = new (std::nothrow) float4[n];
    if (!h0 || !h1) {
        delete[] h0;
        delete[] h1;
        return SPL_ENOMEM;
    }
    int rc = cuda_status(cudaStreamSynchronize(c->stream));
    // the two halves of the 32-byte records into two host arrays (pitched copies)
    if (rc == SPL_OK)
        rc = cuda_status(cudaMemcpy2D(h0, sizeof(float4), &c->recs.p->r0, sizeof(Rec), sizeof(float4),
                                      (size_t)n, cudaMemcpyDeviceToHost));
    if (rc == SPL_OK)
        rc = cuda_status(cudaMemcpy2D(h1, sizeof(float4), &c->recs.p->r1, sizeof(Rec), sizeof(float4),
                                      (size_t)n, cudaMemcpyDeviceToHost));
    if (rc == SPL_OK) {
        const double rs2 = (double)(float)(c->par.r_sml * c->par.r_sml);
        const double rm2 = (double)(float)(c->par.r_small * c->par.r_small);
        const double rl2 = (double)(float)(c->par.r_large * c->par.r_large);
        for (int64_t i = 0; i < n; ++i) {
            uint32_t bits;
            std::memcpy(&bits, &h0[i].x, 4);
            const int xi = (int)(int16_t)(bits & 0xFFFFu), yi = ((int32_t)bits) >> 16;
            const float r2 = h1[i].x;
            if (xs) xs[i] = r2 < 0 ? 0.0 : (double)xi + (double)h0[i].y;
            if (ys) ys[i] = r2 < 0 ? 0.0 : (double)yi + (double)h0[i].z;
            if (r) r[i] = r2 < 0 ? 0.f : std::sqrt(r2);
            if (e) {
                e[3 * i] = h1[i].y;
                e[3 * i + 1] = h1[i].z;
                e[3 * i + 2] = h1[i].w;
            }
            if (cls)
                cls[i] = r2 < 0 ? CLS_INACTIVE
                                : (r2 <= rs2 ? CLS_POINT
                                             : (r2 <= rm2 ? CLS_SMALL : (r2 <= rl2 ? CLS_MEDIUM : CLS_LARGE)));
        }
    }
    delete[] h0;
    delete[] h1;
    return rc;
}

extern "C" int spl_count_work(spl_ctx *c, int64_t out[4]) {
    if (!c || !out) return SPL_EINVAL;
    if (!c->have_particles || !c->have_cam || c->npal < 1) return SPL_ESTATE;
    DeviceGuard g(c->device);
    Views vs{};
    float *no_image = nullptr;
    SPL_TRY(prepare_views(c, &c->cam, 1, &no_image, vs));
    DevBuf<unsigned long long> work;
    SPL_TRY(work.ensure(4));
    int rc = SPL_OK;
    cudaStream_t s = c->stream;
    rc = cuda_status(cudaMemsetAsync(work.p, 0, 4 * sizeof(unsigned long long), s));
    if (rc == SPL_OK) {
        const bool timing = c->timing;
        c->timing = false;
        enqueue_binning(c, vs, s);
        c->timing = timing;
        launch_count_work(c->h_fcs[0], c->recs.p, c->n, work.p, c->sms, s);
        unsigned long long h[4] = {0, 0, 0, 0};
        rc = cuda_status(cudaGetLastError());
        if (rc == SPL_OK) rc = cuda_status(cudaMemcpyAsync(h, work.p, sizeof(h), cudaMemcpyDeviceToHost, s));
        if (rc == SPL_OK) rc = cuda_status(cudaStreamSynchronize(s));
        for (int k = 0; k < 4; ++k) out[k] = (int64_t)h[k];
    }
    work.release();
    return rc;
}

// ---------------------------------------------------------------------------
// spl_render_noalloc: the render for callers that cannot let a library
// allocate device memory -- an application whose device memory comes from
// its own allocator or a fixed budget, or a host program that hands us only
// its own buffers.  The same kernels as spl_render run, but every scratch
// buffer is carved from the file-scope device array below, whose size is
// fixed when the library is loaded; every GPU that loads the library keeps it
// until the process exits.
// ---------------------------------------------------------------------------
namespace {
constexpr int64_t kNaMaxParticles = 131072;
constexpr int kNaMaxTiles = 16384;
constexpr int64_t kNaMaxEntries = 2097152;
constexpr int kNaMaxItems = 32768;

constexpr size_t na_round(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr size_t kNaStats = 0;
constexpr size_t kNaPal = kNaStats + na_round(sizeof(DevStats));
constexpr size_t kNaRecs = kNaPal + na_round(sizeof(float) * 3 * kMaxPalette);
constexpr size_t kNaLarge = kNaRecs + na_round(sizeof(Rec) * kNaMaxParticles);
constexpr size_t kNaCounts = kNaLarge + na_round(sizeof(unsigned) * kNaMaxParticles);
constexpr size_t kNaOffsets = kNaCounts + na_round(sizeof(int) * NLIST * kNaMaxTiles);
constexpr size_t kNaCursor = kNaOffsets + na_round(sizeof(long long) * (NLIST * kNaMaxTiles + 1));
constexpr size_t kNaItemCounts = kNaCursor + na_round(sizeof(long long) * NLIST * kNaMaxTiles);
constexpr size_t kNaItemOffsets = kNaItemCounts + na_round(sizeof(int) * 2 * kNaMaxTiles);
constexpr size_t kNaOvf = kNaItemOffsets + na_round(sizeof(int) * (2 * kNaMaxTiles + 1));
constexpr size_t kNaCtab = kNaOvf + na_round(sizeof(int) * NLIST * kNaMaxTiles);
constexpr size_t kNaEntries = kNaCtab + na_round(sizeof(int2) * ctab_entries(kNaMaxParticles, 1));
constexpr size_t kNaItems = kNaEntries + na_round(sizeof(unsigned) * kNaMaxEntries);
constexpr size_t kNaView = kNaItems + na_round(sizeof(WorkItem) * kNaMaxItems);
constexpr size_t kNaImage = kNaView + na_round(sizeof(FrameConst));
constexpr size_t kNaBytes = kNaImage + na_round(sizeof(float *));
}  // namespace

static_assert(kNaBytes < ((size_t)17 << 20), "the fixed scratch stays below 17 MiB");

// The scratch itself (about 16 MiB as laid out above).  In host
// code this name is only a host-side stand-in; its device address comes from
// cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char spl_noalloc_scratch[kNaBytes];

namespace {
constexpr int kNaMaxDevices = 64;
unsigned char *g_na_scratch[kNaMaxDevices] = {};

// Device address of the scratch on `device` (which must be current); looked
// up on the first call for that device.
int na_scratch(int device, unsigned char **out) {
    if (device < 0 || device >= kNaMaxDevices) return SPL_EINVAL;
    if (!g_na_scratch[device]) {
        void *ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, spl_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            cudaGetLastError();
            return SPL_ECUDA;
        }
        g_na_scratch[device] = static_cast<unsigned char *>(ptr);
    }
    *out = g_na_scratch[device];
    return SPL_OK;
}
}  // namespace

extern "C" int spl_render_noalloc(const spl_particles *p, const spl_camera *cam,
                                  const spl_params *q, const float *rgb, int32_t npal, float s_min,
                                  float s_max, float *d_image, int32_t device, void *stream) {
    if (!p || !cam || !rgb || !d_image || p->n < 0) return SPL_EINVAL;
    if (p->mem_space != SPL_MEM_DEVICE) return SPL_EINVAL;
    if (p->attr_type < SPL_ATTR_F32 || p->attr_type > SPL_ATTR_LOGH16) return SPL_EINVAL;
    if (p->attr_type == SPL_ATTR_LOGH16 && !std::isfinite(p->h_log2_min)) return SPL_EINVAL;
    if (p->n > 0 && (!p->x || !p->y || !p->z || !p->h || !p->I || !p->s)) return SPL_EINVAL;
    if (((p->cr != nullptr) + (p->cg != nullptr) + (p->cb != nullptr)) % 3) return SPL_EINVAL;
    if (!camera_ok(cam)) return SPL_EINVAL;
    if (npal < 1 || npal > kMaxPalette || !std::isfinite(s_min) || !std::isfinite(s_max))
        return SPL_EINVAL;
    for (int k = 0; k < 3 * npal; ++k)
        if (!std::isfinite(rgb[k])) return SPL_EINVAL;
    spl_ctx tmp;   // parameters only; none of its buffers is allocated
    if (q) {
        if (!params_ok(q) || q->mode == SPL_MODE_ABSORB) return SPL_EINVAL;
        tmp.par = *q;
    } else {
        spl_default_params(&tmp.par);
    }
    tmp.npal = npal;
    tmp.s_min = s_min;
    tmp.s_max = s_max;
    const FrameConst fc = make_frame(&tmp, *cam);
    if (p->n > kNaMaxParticles || fc.ntiles > kNaMaxTiles) return SPL_ELIMIT;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        return SPL_ECUDA;
    }
    if (device < 0 || device >= ndev) return SPL_EINVAL;
    DeviceGuard g(device);
    cudaStream_t s = (cudaStream_t)stream;
    // the call waits on the host mid-way, which a capturing stream forbids
    cudaStreamCaptureStatus capturing = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &capturing) != cudaSuccess) {
        cudaGetLastError();
        return SPL_ECUDA;
    }
    if (capturing != cudaStreamCaptureStatusNone) return SPL_ESTATE;
    unsigned char *base = nullptr;
    SPL_TRY(na_scratch(device, &base));
    DevStats *dst = reinterpret_cast<DevStats *>(base + kNaStats);
    float *pal = reinterpret_cast<float *>(base + kNaPal);
    Rec *recs = reinterpret_cast<Rec *>(base + kNaRecs);
    unsigned *large_ids = reinterpret_cast<unsigned *>(base + kNaLarge);
    int *counts = reinterpret_cast<int *>(base + kNaCounts);
    long long *offsets = reinterpret_cast<long long *>(base + kNaOffsets);
    long long *cursor = reinterpret_cast<long long *>(base + kNaCursor);
    int *item_counts = reinterpret_cast<int *>(base + kNaItemCounts);
    int *item_offsets = reinterpret_cast<int *>(base + kNaItemOffsets);
    int *ovf = reinterpret_cast<int *>(base + kNaOvf);
    int2 *ctab = reinterpret_cast<int2 *>(base + kNaCtab);
    unsigned *entries = reinterpret_cast<unsigned *>(base + kNaEntries);
    WorkItem *items = reinterpret_cast<WorkItem *>(base + kNaItems);
    FrameConst *d_fc = reinterpret_cast<FrameConst *>(base + kNaView);
    float **d_img = reinterpret_cast<float **>(base + kNaImage);
    int sms = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    FrameConst fcv = fc;
    fcv.view = 0;
    fcv.tile_base = 0;
    fcv.slot_base = 0;
    fcv.rec_base = 0;
    Views vs{};
    vs.fcs = d_fc;
    vs.nviews = 1;
    vs.total_tiles = fc.ntiles;
    vs.tile = fc.tile;
    vs.n = p->n;

    // the array keeps the previous call's contents: clear what starts at zero
    // (the error word stays: the previous call's passes may have set it, and
    // it is read at this call's synchronisation point)
    SPL_CUDA(cudaMemcpyAsync(pal, rgb, sizeof(float) * 3 * npal, cudaMemcpyHostToDevice, s));
    SPL_CUDA(cudaMemcpyAsync(d_fc, &fcv, sizeof(FrameConst), cudaMemcpyHostToDevice, s));
    SPL_CUDA(cudaMemcpyAsync(d_img, &d_image, sizeof(float *), cudaMemcpyHostToDevice, s));
    SPL_CUDA(cudaMemsetAsync(dst, 0, offsetof(DevStats, err), s));
    SPL_CUDA(cudaMemsetAsync(counts, 0, sizeof(int) * NLIST * fc.ntiles, s));
    SPL_CUDA(cudaMemsetAsync(ovf, 0, sizeof(int) * NLIST * fc.ntiles, s));
    RasterArgs ra{};
    ra.n = p->n;
    ra.x = p->x; ra.y = p->y; ra.z = p->z;
    ra.h = p->h; ra.I = p->I; ra.s = p->s;
    ra.cr = p->cr; ra.cg = p->cg; ra.cb = p->cb;
    ra.h_log2_min = p->h_log2_min;
    ra.pal = pal;
    ra.recs = recs;
    ra.counts = counts;
    ra.ovf = ovf;
    ra.ctab = ctab;
    ra.large_ids = large_ids;
    ra.st = dst;
    launch_raster(vs, ra, p->attr_type, s);
    BinArgs ba{};
    ba.recs = recs;
    ba.large_ids = large_ids;
    ba.counts = counts;
    ba.ovf = ovf;
    ba.offsets = offsets;
    ba.ctab = ctab;
    ba.cursor = cursor;
    ba.st = dst;
    launch_count_large(vs, ba, sms, s);
    launch_slot_offsets(NLIST * fc.ntiles, counts, ovf, offsets, cursor, &dst->slot_total, s);
    launch_item_counts(vs, offsets, item_counts, dst, s);
    launch_scan(2 * fc.ntiles, item_counts, item_offsets, nullptr, 2, dst->item_totals, s);
    SPL_CUDA(cudaGetLastError());
    DevStats h;
    SPL_CUDA(cudaMemcpyAsync(&h, dst, sizeof(DevStats), cudaMemcpyDeviceToHost, s));
    SPL_CUDA(cudaStreamSynchronize(s));
    if (h.err) {
        // a check failed in this binning or in the previous call's passes
        SPL_CUDA(cudaMemsetAsync(&dst->err, 0, sizeof(unsigned), s));
        return SPL_EDEVICE;
    }
    const int64_t total = h.slot_total;
    const int n_tile_items = h.item_totals[0], n_large_items = h.item_totals[1];
    if (total > kNaMaxEntries || (int64_t)n_tile_items + n_large_items > kNaMaxItems)
        return SPL_ELIMIT;
    launch_zero_images(vs, d_img, sms, s);
    ba.entries = entries;
    ba.entries_cap = kNaMaxEntries;
    launch_scatter(vs, ba, sms, s);
    launch_fill_items(vs, offsets, item_offsets, items, kNaMaxItems, dst, s);
    TileArgs ta{};
    ta.recs = recs;
    ta.offsets = offsets;
    ta.entries = entries;
    ta.items = items;
    ta.items_cap = kNaMaxItems;
    ta.images = d_img;
    ta.st = dst;
    launch_tile_pass(vs, ta, sms, s);
    if (n_large_items > 0) launch_large_pass(vs, ta, sms, s);
    if (tmp.par.mode == SPL_MODE_EA) launch_epilogue_views(vs, d_img, sms, s);
    SPL_CUDA(cudaGetLastError());
    return SPL_OK;
}
