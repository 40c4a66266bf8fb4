// gsrf_api.cu -- the extern "C" boundary of libgsrf.so (declared in include/gsrf.h):
// argument checks, workspace layout, and the launch sequences of each call.
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <unordered_map>

#include "gsrf_internal.cuh"

namespace gsrf {

static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

bool make_layout(const gsrf_plan* p, Layout* L) {
    const gsrf_grid& g = p->grid;
    L->ntu = (g.n_az + g.tile_w - 1) / g.tile_w;
    L->ntv = (g.n_el + g.tile_h - 1) / g.tile_h;
    L->n_tiles = L->ntu * L->ntv;
    L->n_rx = p->n_rx;
    L->n = p->n_gauss;
    L->cap = p->pair_capacity;
    L->dchunks = (int32_t)((p->n_gauss + kDChunk - 1) / kDChunk);
    L->echunks = (int32_t)((p->n_gauss + kEChunk - 1) / kEChunk);
    L->pchunks_max = (p->pair_capacity + kChunk - 1) / kChunk + p->n_rx;
    const size_t n = (size_t)p->n_gauss, nr = (size_t)p->n_rx, cap = (size_t)p->pair_capacity;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes);
        return o;
    };
    L->status = take(sizeof(DevStatus));
    L->rxpos = take(nr * 3 * sizeof(float));
    L->txpos = take(3 * sizeof(float));
    L->gacc = take(n * grad_floats(plan_degree(p)) * sizeof(float));
    L->raytab = take((size_t)g.n_az * g.n_el * raytab_floats(plan_degree(p)) * sizeof(float));
    // the ray table's per-column and per-row FP64 factors: (cos, sin)(m az) for m = 1..5,
    // sin el, cos el and P_l^m (m <= l <= 5)
    L->rayfac = take(((size_t)g.n_az * 2 * kMaxDegree + (size_t)g.n_el * (2 + (kMaxDegree + 1) * (kMaxDegree + 2) / 2)) * sizeof(double));
    L->fle = take(n * fle_floats(plan_degree(p)) * sizeof(float));
    L->gshape = take(n * sizeof(GShape));
    L->dpath = take(n * sizeof(double));
    L->view = take(nr * n * sizeof(View));
    L->cover = take(nr * n * sizeof(Cover));
    L->dkey = take(nr * n * 4);
    L->dkey2 = take(nr * n * 4);
    L->dval = take(nr * n * 4);
    L->dval2 = take(nr * n * 4);
    L->dhist = take(nr * (size_t)L->dchunks * 256 * 4);
    L->dvis = take(nr * 4);
    L->dchunk_sum = take(nr * (size_t)L->echunks * 4);
    L->egroup = take(nr * (size_t)L->echunks * (kEChunk / 32) * 4);
    L->eslice = take(((size_t)L->n_rx + 1) * 4);
    L->rx_base = take((nr + 1) * 8);
    L->rx_total = take(nr * 4);
    L->pchunk_base = take((nr + 1) * 4);
    L->pkeys = take(cap * 8);
    L->pkeys2 = take(cap * 4);  // the pairs' tile indices in depth order (the tile sort's input)
    L->pids = take(cap * 4);
    L->pids2 = take(cap * 4);
    L->tile_start = take(nr * (size_t)(L->n_tiles + 1) * 4);
    L->thist = take((size_t)L->pchunks_max * L->n_tiles * 4);
    // the render's work queue: one item per (receiver, tile, ray block, subcarrier chunk);
    // chunks of 8 subcarriers are the most any launch uses
    const size_t items = nr * (size_t)L->n_tiles * (size_t)(g.tile_w * g.tile_h / 32) * (size_t)((p->n_f + 7) / 8);
    L->qkeys = take(items * 4);
    L->qkeys2 = take(items * 4);
    L->qorder = take(items * 4);
    L->qhist = take((items + kSmallChunk - 1) / kSmallChunk * 32 * 4);
    L->qcounter = take(8);
    // the paper's splatting circles, per (receiver, Gaussian), only for that variant
    L->circle = take((p->variant & GSRF_VARIANT_PAPER_CULLING) ? nr * n * sizeof(float4) : 0);
    // the t_mid-order variant's per-ray hit keys
    L->tbuf = take((p->variant & GSRF_VARIANT_ORDER_T_MID) ? nr * (size_t)g.n_az * g.n_el * kOrderCap * 8 : 0);
    L->total = off;
    return true;
}

// ---------------------------------------------------------------------------
// Stage timers (gsrf_stage_times): per workspace, a start and an end CUDA event per
// stage, recorded on the caller's stream around the stage's launches.  Host-side state
// only (events, no device memory); a stream that is capturing records nothing.
// ---------------------------------------------------------------------------
constexpr int kStages = 8;
constexpr size_t kMaxTimedWorkspaces = 1024;

struct StageEvents {
    int device = -1;
    cudaEvent_t ev[2 * kStages] = {};
    bool done[kStages] = {};
};

static std::mutex g_stage_mu;
static std::unordered_map<const void*, StageEvents> g_stage;

static void destroy_events(StageEvents& e) {
    for (int i = 0; i < 2 * kStages; ++i)
        if (e.ev[i]) cudaEventDestroy(e.ev[i]);
    e = StageEvents();
}

// The events of (workspace, stage) ready to record on `st`, or null when the stream is
// capturing or an event cannot be had (timing is then simply not kept).
static StageEvents* stage_slot(const void* ws, cudaStream_t st) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return nullptr;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    auto it = g_stage.find(ws);
    if (it == g_stage.end()) {
        if (g_stage.size() >= kMaxTimedWorkspaces) {  // forget the oldest-inserted bucket entry
            destroy_events(g_stage.begin()->second);
            g_stage.erase(g_stage.begin());
        }
        it = g_stage.emplace(ws, StageEvents()).first;
    }
    StageEvents& e = it->second;
    if (e.device != dev) {
        destroy_events(e);
        e.device = dev;
        for (int i = 0; i < 2 * kStages; ++i) {
            if (cudaEventCreate(&e.ev[i]) != cudaSuccess) {
                cudaGetLastError();
                destroy_events(e);
                return nullptr;
            }
        }
    }
    return &e;
}

// Records the start of `stage` on construction and its end on destruction.
struct StageTimer {
    StageEvents* e = nullptr;
    int stage;
    cudaStream_t st;
    StageTimer(const void* ws, int stage_, cudaStream_t st_) : stage(stage_), st(st_) {
        std::lock_guard<std::mutex> lock(g_stage_mu);
        e = stage_slot(ws, st);
        if (e && cudaEventRecord(e->ev[2 * stage], st) != cudaSuccess) {
            cudaGetLastError();
            e = nullptr;
        }
    }
    ~StageTimer() {
        if (!e) return;
        std::lock_guard<std::mutex> lock(g_stage_mu);
        e->done[stage] = cudaEventRecord(e->ev[2 * stage + 1], st) == cudaSuccess;
        if (!e->done[stage]) cudaGetLastError();
    }
};

}  // namespace gsrf

using namespace gsrf;

static gsrf_status check_grid(const gsrf_grid* g) {
    if (!g) return GSRF_ERR_INVALID_ARG;
    if (g->n_az < 1 || g->n_el < 1 || g->n_az > 65536 || g->n_el > 65536) return GSRF_ERR_INVALID_ARG;
    if (!(g->daz_deg > 0.0f) || !(g->del_deg > 0.0f)) return GSRF_ERR_INVALID_ARG;
    if (!(g->az0_deg >= -360.0f && g->az0_deg <= 360.0f)) return GSRF_ERR_INVALID_ARG;
    if (!(g->el0_deg >= -90.0f && g->el0_deg <= 90.0f)) return GSRF_ERR_INVALID_ARG;
    if (!(g->r_rx >= 0.0f) || !(g->eps_T >= 0.0f && g->eps_T < 1.0f)) return GSRF_ERR_INVALID_ARG;
    if (!(g->alpha_max > 0.0f && g->alpha_max < 1.0f)) return GSRF_ERR_INVALID_ARG;
    const bool tw_ok = g->tile_w == 8 || g->tile_w == 16 || g->tile_w == 32;
    const bool th_ok = g->tile_h == 4 || g->tile_h == 8 || g->tile_h == 16 || g->tile_h == 32;
    if (!tw_ok || !th_ok || g->tile_w * g->tile_h < 32) return GSRF_ERR_UNSUPPORTED;
    const int ntu = (g->n_az + g->tile_w - 1) / g->tile_w, ntv = (g->n_el + g->tile_h - 1) / g->tile_h;
    if (ntu > 64 || ntu * ntv > kMaxTiles) return GSRF_ERR_UNSUPPORTED;
    return GSRF_OK;
}

static gsrf_status check_plan(const gsrf_plan* p) {
    if (!p) return GSRF_ERR_INVALID_ARG;
    if (p->n_gauss < 0 || p->n_gauss >= (1ll << 31)) return GSRF_ERR_INVALID_ARG;
    if (p->n_rx < 1 || p->n_rx > 65535) return GSRF_ERR_INVALID_ARG;
    if (p->n_f < 1 || p->n_f > kMaxNf) return GSRF_ERR_INVALID_ARG;
    if (!(p->f0_hz > 0.0) || !(p->df_hz >= 0.0)) return GSRF_ERR_INVALID_ARG;
    if (p->pair_capacity < 0 || p->pair_capacity > (1ll << 40)) return GSRF_ERR_INVALID_ARG;
    if ((size_t)p->n_gauss * (size_t)p->n_rx >= (1ull << 40)) return GSRF_ERR_INVALID_ARG;
    const int bw = p->ray_block_w;
    if (!(bw == 0 || bw == 4 || bw == 8 || bw == 16 || bw == 32)) return GSRF_ERR_INVALID_ARG;
    if (!(p->stage == 0 || p->stage == 16 || p->stage == 32)) return GSRF_ERR_INVALID_ARG;
    if (p->ckpt_every < 0 || p->ckpt_every % 32 != 0 || p->ckpt_every > (1 << 24)) return GSRF_ERR_INVALID_ARG;
    if (p->ckpt_every > 0 && (p->ckpt_slots < 1 || p->ckpt_slots > 64)) return GSRF_ERR_INVALID_ARG;
    if (p->variant < 0 || p->variant > 31) return GSRF_ERR_INVALID_ARG;
    if ((p->variant & GSRF_VARIANT_ORDER_T_MID) &&
        (p->n_f > 1 || plan_degree(p) != 3 || (p->variant & GSRF_VARIANT_PATH_AT_REP)))
        return GSRF_ERR_UNSUPPORTED;  // its kernel instance: one frequency, L = 3
    if ((p->variant & GSRF_VARIANT_PATH_AT_REP) && (p->n_f > 1 || plan_degree(p) != 3))
        return GSRF_ERR_UNSUPPORTED;  // its kernel instance: one frequency, L = 3
    if (p->fle_degree < 0 || p->fle_degree > kMaxDegree) return GSRF_ERR_INVALID_ARG;
    if (plan_degree(p) != 3 && (p->n_f > 1 || (p->variant & GSRF_VARIANT_RADIANCE_AT_MEAN)))
        return GSRF_ERR_UNSUPPORTED;  // other degrees: one frequency, radiance per ray
    const gsrf_status s = check_grid(&p->grid);
    if (s != GSRF_OK) return s;
    const int w = plan_block_w(p);
    if (p->grid.tile_w % w != 0 || p->grid.tile_h % (32 / w) != 0) return GSRF_ERR_UNSUPPORTED;
    return GSRF_OK;
}

static gsrf_status check_ws(const gsrf_plan* p, const void* ws, size_t ws_bytes, Layout* L) {
    gsrf_status s = check_plan(p);
    if (s != GSRF_OK) return s;
    make_layout(p, L);
    if (!ws || ((uintptr_t)ws & 255) != 0 || ws_bytes < L->total) return GSRF_ERR_INVALID_ARG;
    return GSRF_OK;
}

static gsrf_status check_gauss(const gsrf_plan* p, const gsrf_gaussians* g) {
    if (!g || g->n != p->n_gauss) return GSRF_ERR_INVALID_ARG;
    if (g->n > 0 && (!g->means || !g->log_scales || !g->quats || !g->opacity_logit || !g->coeffs))
        return GSRF_ERR_INVALID_ARG;
    if (((uintptr_t)g->coeffs & 15) != 0) return GSRF_ERR_INVALID_ARG;  // staged as float4
    return GSRF_OK;
}

static gsrf_status cuda_status(cudaError_t e) { return e == cudaSuccess ? GSRF_OK : GSRF_ERR_CUDA; }

extern "C" {

const char* gsrf_version(void) { return "gsrf-gb300 0.1 (sm_103a)"; }

gsrf_status gsrf_workspace_size(const gsrf_plan* plan, size_t* bytes) {
    gsrf_status s = check_plan(plan);
    if (s != GSRF_OK) return s;
    if (!bytes) return GSRF_ERR_INVALID_ARG;
    Layout L;
    make_layout(plan, &L);
    *bytes = L.total;
    return GSRF_OK;
}

gsrf_status gsrf_workspace_layout(const gsrf_plan* plan, gsrf_layout* out) {
    gsrf_status s = check_plan(plan);
    if (s != GSRF_OK) return s;
    if (!out) return GSRF_ERR_INVALID_ARG;
    Layout L;
    make_layout(plan, &L);
    out->pair_keys = L.pkeys;
    out->pair_ids = L.pids;
    out->rx_pair_base = L.rx_base;
    out->tile_start = L.tile_start;
    out->status = L.status;
    out->n_tiles_u = L.ntu;
    out->n_tiles_v = L.ntv;
    out->view = L.view;
    return GSRF_OK;
}

size_t gsrf_ray_state_bytes(const gsrf_plan* plan) {
    if (check_plan(plan) != GSRF_OK) return 0;
    const size_t rays = (size_t)plan->n_rx * plan->grid.n_az * plan->grid.n_el;
    return rays * sizeof(RayState) + (plan->ckpt_every > 0 ? rays * (size_t)plan->ckpt_slots * sizeof(float4) : 0);
}

gsrf_status gsrf_project(const gsrf_plan* plan, const gsrf_gaussians* g, const float* rx_pos,
                         const float* tx_pos, void* workspace, size_t ws_bytes, void* stream) {
    Layout L;
    gsrf_status s = check_ws(plan, workspace, ws_bytes, &L);
    if (s != GSRF_OK) return s;
    if ((s = check_gauss(plan, g)) != GSRF_OK) return s;
    if (!rx_pos || !tx_pos) return GSRF_ERR_INVALID_ARG;
    StageTimer tm(workspace, GSRF_STAGE_PROJECT, (cudaStream_t)stream);
    return cuda_status(launch_project(plan, L, g, rx_pos, tx_pos, workspace, (cudaStream_t)stream));
}

gsrf_status gsrf_bin(const gsrf_plan* plan, void* workspace, size_t ws_bytes, void* stream) {
    Layout L;
    gsrf_status s = check_ws(plan, workspace, ws_bytes, &L);
    if (s != GSRF_OK) return s;
    StageTimer tm(workspace, GSRF_STAGE_BIN, (cudaStream_t)stream);
    return cuda_status(launch_bin(plan, L, workspace, (cudaStream_t)stream));
}

gsrf_status gsrf_pair_keys(const gsrf_plan* plan, void* workspace, size_t ws_bytes, void* stream) {
    Layout L;
    gsrf_status s = check_ws(plan, workspace, ws_bytes, &L);
    if (s != GSRF_OK) return s;
    return cuda_status(launch_pair_keys(L, workspace, (cudaStream_t)stream));
}

gsrf_status gsrf_render_fwd(const gsrf_plan* plan, const gsrf_gaussians* g, void* workspace, size_t ws_bytes,
                            float* out_rays, void* ray_state, void* stream) {
    Layout L;
    gsrf_status s = check_ws(plan, workspace, ws_bytes, &L);
    if (s != GSRF_OK) return s;
    if ((s = check_gauss(plan, g)) != GSRF_OK) return s;
    if (!out_rays || ((uintptr_t)out_rays & 7) != 0 || ((uintptr_t)ray_state & 15) != 0)
        return GSRF_ERR_INVALID_ARG;
    StageTimer tm(workspace, GSRF_STAGE_RENDER_FWD, (cudaStream_t)stream);
    return cuda_status(launch_render_fwd(plan, L, g, workspace, out_rays, ray_state, (cudaStream_t)stream));
}

gsrf_status gsrf_render_bwd(const gsrf_plan* plan, const gsrf_gaussians* g, void* workspace, size_t ws_bytes,
                            const void* ray_state, const float* grad_rays, float* g_means, float* g_log_scales,
                            float* g_quats, float* g_opacity_logit, float* g_coeffs, float* g_phase_b,
                            void* stream) {
    Layout L;
    gsrf_status s = check_ws(plan, workspace, ws_bytes, &L);
    if (s != GSRF_OK) return s;
    if ((s = check_gauss(plan, g)) != GSRF_OK) return s;
    if (!ray_state || !grad_rays || ((uintptr_t)ray_state & 15) != 0 || ((uintptr_t)grad_rays & 7) != 0)
        return GSRF_ERR_INVALID_ARG;
    if ((plan->variant & ~(GSRF_VARIANT_NORMALISED_WEIGHT | GSRF_VARIANT_PAPER_CULLING)) != 0)
        return GSRF_ERR_UNSUPPORTED;  // the default reading, normalised weight, circle culling (any degree)
    StageTimer tm(workspace, GSRF_STAGE_RENDER_BWD, (cudaStream_t)stream);
    return cuda_status(launch_render_bwd(plan, L, g, workspace, ray_state, grad_rays, g_means, g_log_scales, g_quats,
                                         g_opacity_logit, g_coeffs, g_phase_b, (cudaStream_t)stream));
}

gsrf_status gsrf_render(const gsrf_plan* plan, const gsrf_gaussians* g, const float* rx_pos, const float* tx_pos,
                        void* workspace, size_t ws_bytes, float* out_rays, void* ray_state, void* stream) {
    gsrf_status s = gsrf_project(plan, g, rx_pos, tx_pos, workspace, ws_bytes, stream);
    if (s != GSRF_OK) return s;
    if ((s = gsrf_bin(plan, workspace, ws_bytes, stream)) != GSRF_OK) return s;
    return gsrf_render_fwd(plan, g, workspace, ws_bytes, out_rays, ray_state, stream);
}

gsrf_status gsrf_batch_workspace_size(int32_t n_jobs, const gsrf_plan* plans, size_t* bytes) {
    if (n_jobs < 1 || n_jobs > GSRF_MAX_BATCH_JOBS || !plans || !bytes) return GSRF_ERR_INVALID_ARG;
    for (int j = 0; j < n_jobs; ++j) {
        gsrf_status s = check_plan(&plans[j]);
        if (s != GSRF_OK) return s;
        if (plans[j].n_f != 1) return GSRF_ERR_UNSUPPORTED;
    }
    *bytes = batch_workspace_bytes(n_jobs, plans);
    return GSRF_OK;
}

gsrf_status gsrf_render_batch(int32_t n_jobs, const gsrf_plan* plans, void* const* workspaces, const size_t* ws_bytes,
                              float* const* outs, void* batch_ws, size_t batch_ws_bytes, uint64_t* job_done_ns,
                              int32_t flags, void* stream) {
    size_t need = 0;
    gsrf_status s = gsrf_batch_workspace_size(n_jobs, plans, &need);
    if (s != GSRF_OK) return s;
    if (!workspaces || !ws_bytes || !outs || !batch_ws || ((uintptr_t)batch_ws & 255) != 0 || batch_ws_bytes < need)
        return GSRF_ERR_INVALID_ARG;
    for (int j = 0; j < n_jobs; ++j) {
        Layout L;
        if ((s = check_ws(&plans[j], workspaces[j], ws_bytes[j], &L)) != GSRF_OK) return s;
        if (!outs[j] || ((uintptr_t)outs[j] & 7) != 0) return GSRF_ERR_INVALID_ARG;
        if (plan_degree(&plans[j]) != 3 || (plans[j].variant & (GSRF_VARIANT_PATH_AT_REP | GSRF_VARIANT_ORDER_T_MID)))
            return GSRF_ERR_UNSUPPORTED;
    }
    if (((uintptr_t)job_done_ns & 7) != 0 || (flags & ~GSRF_BATCH_JOB_ORDER) != 0) return GSRF_ERR_INVALID_ARG;
    if (batch_items(n_jobs, plans) >= (1ll << 32)) return GSRF_ERR_UNSUPPORTED;  // 32-bit item ids
    StageTimer tm(batch_ws, GSRF_STAGE_BATCH, (cudaStream_t)stream);
    return cuda_status(launch_render_batch(n_jobs, plans, workspaces, outs, batch_ws,
                                           reinterpret_cast<unsigned long long*>(job_done_ns),
                                           (flags & GSRF_BATCH_JOB_ORDER) != 0, (cudaStream_t)stream));
}

gsrf_status gsrf_received_signal(const float* rays, int32_t n_rx, int32_t n_f, int32_t n_el, int32_t n_az,
                                 int32_t mode, float* out, void* stream) {
    if (!rays || !out || n_rx < 1 || n_f < 1 || n_el < 1 || n_az < 1 || mode < 0 || mode > 3)
        return GSRF_ERR_INVALID_ARG;
    if ((size_t)n_rx * n_f > 0x0fffffffu || (size_t)n_el * n_az > 0x7fffffffu) return GSRF_ERR_INVALID_ARG;
    return cuda_status(launch_signal(rays, n_rx, n_f, n_el, n_az, mode, out, (cudaStream_t)stream));
}

gsrf_status gsrf_read_status(const void* workspace, size_t ws_bytes, gsrf_run_status* out, void* stream) {
    if (!workspace || !out || ws_bytes < sizeof(DevStatus)) return GSRF_ERR_INVALID_ARG;
    DevStatus h;
    cudaError_t e = cudaMemcpyAsync(&h, workspace, sizeof(h), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return GSRF_ERR_CUDA;
    out->code = h.code;
    out->first_bad = h.first_bad == 0x7fffffff ? -1 : h.first_bad;
    out->required_pairs = h.required_pairs;
    for (int i = 0; i < 4; ++i) out->stats[i] = (int64_t)h.stats[i];
    return GSRF_OK;
}

gsrf_status gsrf_stage_times(const void* workspace, float* ms) {
    if (!workspace || !ms) return GSRF_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_stage_mu);
    auto it = g_stage.find(workspace);
    if (it == g_stage.end()) return GSRF_ERR_INVALID_ARG;
    const StageEvents& e = it->second;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GSRF_ERR_CUDA;
    if (dev != e.device && cudaSetDevice(e.device) != cudaSuccess) return GSRF_ERR_CUDA;
    gsrf_status s = GSRF_OK;
    for (int i = 0; i < kStages; ++i) {
        ms[i] = -1.0f;
        if (!e.done[i]) continue;
        float t = 0.0f;
        if (cudaEventSynchronize(e.ev[2 * i + 1]) != cudaSuccess ||
            cudaEventElapsedTime(&t, e.ev[2 * i], e.ev[2 * i + 1]) != cudaSuccess) {
            cudaGetLastError();
            s = GSRF_ERR_CUDA;
            continue;
        }
        ms[i] = t;
    }
    if (dev != e.device) cudaSetDevice(dev);
    return s;
}

}  // extern "C"
