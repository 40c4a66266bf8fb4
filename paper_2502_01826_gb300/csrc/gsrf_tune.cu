// gsrf_tune.cu -- the autotuner of the work split: tile shape, rays per warp block and
// candidates per shared-memory stage.  None of them changes a result (the render's
// arithmetic per ray is the same under every split); they change how well the list
// walks, the staging and the work queue fit the scene.  The tuner measures the
// caller's own problem on the caller's stream, so the choice reflects the scene's
// depth structure, the receivers' positions and the grid, not a model of them.
#include <stdio.h>
#include <string.h>

#include <vector>

#include "gsrf_internal.cuh"

namespace gsrf {

// Tile shapes tried: the paper's 16 x 16 and its neighbours with 128 to 1024 rays.
static const int kTileShapes[][2] = {{16, 16}, {32, 8}, {16, 8}, {8, 16}, {32, 16}, {16, 32}, {32, 32}, {8, 8}};
static const int kBlockWidths[] = {4, 8, 16, 32};
static const int kStages[] = {16, 32};

static gsrf_plan with_split(const gsrf_plan& p, int tw, int th, int bw, int stage) {
    gsrf_plan q = p;
    q.grid.tile_w = tw;
    q.grid.tile_h = th;
    q.ray_block_w = bw;
    q.stage = stage;
    return q;
}

// Median of the event-timed durations (ms) of `reps` runs of fn after one untimed run.
template <typename F>
static gsrf_status time_median(F&& fn, int reps, cudaStream_t st, float* ms) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return GSRF_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return GSRF_ERR_CUDA;
    }
    gsrf_status s = fn();
    std::vector<float> t;
    for (int i = 0; i < reps && s == GSRF_OK; ++i) {
        cudaEventRecord(e0, st);
        s = fn();
        cudaEventRecord(e1, st);
        if (s != GSRF_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            s = GSRF_ERR_CUDA;
            break;
        }
        float x = 0.0f;
        cudaEventElapsedTime(&x, e0, e1);
        t.push_back(x);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != GSRF_OK) return s;
    for (size_t i = 1; i < t.size(); ++i)  // insertion sort: a handful of values
        for (size_t j = i; j > 0 && t[j] < t[j - 1]; --j) std::swap(t[j], t[j - 1]);
    *ms = t.empty() ? 0.0f : t[t.size() / 2];
    return GSRF_OK;
}

}  // namespace gsrf

using namespace gsrf;

extern "C" {

gsrf_status gsrf_autotune_workspace_size(const gsrf_plan* plan, size_t* bytes) {
    if (!plan || !bytes) return GSRF_ERR_INVALID_ARG;
    size_t best = 0;
    bool any = false;
    for (const auto& ts : kTileShapes) {
        size_t b = 0;
        const gsrf_plan q = with_split(*plan, ts[0], ts[1], 0, 0);
        if (gsrf_workspace_size(&q, &b) == GSRF_OK) {
            any = true;
            best = b > best ? b : best;
        }
    }
    if (!any) return gsrf_workspace_size(plan, bytes);
    *bytes = best;
    return GSRF_OK;
}

gsrf_status gsrf_autotune(const gsrf_plan* plan, const gsrf_gaussians* g, const float* rx_pos, const float* tx_pos,
                          void* workspace, size_t ws_bytes, float* out_rays, const gsrf_tune_backward* bwd,
                          int32_t reps, gsrf_tune_result* results, int32_t max_results, int32_t* n_results,
                          gsrf_tune_result* best, void* stream) {
    if (!plan || !g || !rx_pos || !tx_pos || !workspace || !out_rays || !best || reps < 1 || reps > 100)
        return GSRF_ERR_INVALID_ARG;
    if (bwd && (!bwd->ray_state || !bwd->grad_rays)) return GSRF_ERR_INVALID_ARG;
    if (bwd && (plan->variant & ~(GSRF_VARIANT_NORMALISED_WEIGHT | GSRF_VARIANT_PAPER_CULLING)) != 0)
        return GSRF_ERR_UNSUPPORTED;  // the readings the backward has
    if (max_results < 0 || (max_results > 0 && !results)) return GSRF_ERR_INVALID_ARG;
    size_t need = 0;
    gsrf_status s = gsrf_workspace_size(plan, &need);  // validates the caller's plan
    if (s != GSRF_OK) return s;
    const cudaStream_t st = (cudaStream_t)stream;
    int n = 0;
    float best_ms = 3.0e38f;
    bool found = false;
    for (const auto& ts : kTileShapes) {
        gsrf_plan q = with_split(*plan, ts[0], ts[1], 0, 0);
        if (gsrf_workspace_size(&q, &need) != GSRF_OK || need > ws_bytes) continue;  // not this grid
        float pb_ms = 0.0f;
        s = time_median([&]() -> gsrf_status {
            gsrf_status r = gsrf_project(&q, g, rx_pos, tx_pos, workspace, ws_bytes, stream);
            return r == GSRF_OK ? gsrf_bin(&q, workspace, ws_bytes, stream) : r;
        }, reps, st, &pb_ms);
        if (s != GSRF_OK) return s;
        gsrf_run_status rs;
        if ((s = gsrf_read_status(workspace, ws_bytes, &rs, stream)) != GSRF_OK) return s;
        if (rs.code != GSRF_OK) continue;  // e.g. more pairs than the plan's capacity
        for (int bw : kBlockWidths) {
            if (ts[0] % bw != 0 || ts[1] % (32 / bw) != 0) continue;
            for (int stg : kStages) {
                const gsrf_plan c = with_split(*plan, ts[0], ts[1], bw, stg);
                float r_ms = 0.0f;
                s = time_median([&]() -> gsrf_status {
                    gsrf_status r = gsrf_render_fwd(&c, g, workspace, ws_bytes, out_rays, bwd ? bwd->ray_state : nullptr,
                                                    stream);
                    if (r != GSRF_OK || !bwd) return r;
                    return gsrf_render_bwd(&c, g, workspace, ws_bytes, bwd->ray_state, bwd->grad_rays, bwd->g_means,
                                           bwd->g_log_scales, bwd->g_quats, bwd->g_opacity_logit, bwd->g_coeffs,
                                           bwd->g_phase_b, stream);
                }, reps, st, &r_ms);
                if (s != GSRF_OK) return s;
                const gsrf_tune_result res = {ts[0], ts[1], bw, stg, pb_ms, r_ms};
                if (n < max_results) results[n] = res;
                ++n;
                if (pb_ms + r_ms < best_ms) {
                    best_ms = pb_ms + r_ms;
                    *best = res;
                    found = true;
                }
            }
        }
    }
    if (n_results) *n_results = n;
    return found ? GSRF_OK : GSRF_ERR_CAPACITY;
}

}  // extern "C"
