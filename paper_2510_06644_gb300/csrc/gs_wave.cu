// Multi-session waves (the serving form): one fused tracking iteration of
// every job of a wave -- projection with the binning's tile rows, column
// scan with the tile scan, key scatter with the heavy-first order, bucket
// sort, forward compositing with the L1 loss (Eq. 6), backward compositing
// (Sec. 2.2 Step 4) and backward projection with the pose step (Step 5) --
// in launches whose grids span all jobs.  Each kernel is the single-session
// kernel's body; a CTA finds its job and its block inside the job in the
// wave's descriptor table (gs_internal.cuh, Wave<J>), which is the launch's
// __grid_constant__ parameter block.  The zeroing the single-session calls
// do with memsets (the loss, the two tickets, the 2D gradients) happens in
// the projection launch.
#include <stdio.h>

#include "gs_internal.cuh"

using namespace gs;

size_t gs_project_bwd_ws(int64_t n);

static gs_status job_checks(const gs_config* cfg, const gs_track_job& j, int i) {
    (void)cfg;
    const gs_camera& c = j.cam;
    if (c.width <= 0 || c.height <= 0 || c.sx < 1 || c.sy < 1 || c.width > (1 << 20) || c.height > (1 << 20))
        return set_error(GS_ERR_INVALID_ARG, "job %d: bad camera size or stride", i);
    if (!(c.fx > 0.f) || !(c.fy > 0.f)) return set_error(GS_ERR_INVALID_ARG, "job %d: focal length must be > 0", i);
    if (j.g.n < 1 || j.g.n > (int64_t)0xFFFFFFF0LL) return set_error(GS_ERR_INVALID_ARG, "job %d: bad Gaussian count", i);
    if (!j.g.means || !j.g.log_scales || !j.g.quats || !j.g.opacity_logit || !j.g.rgb)
        return set_error(GS_ERR_INVALID_ARG, "job %d: a Gaussian parameter array is NULL", i);
    if (!j.splats || ((uintptr_t)j.splats & 15))
        return set_error(GS_ERR_INVALID_ARG, "job %d: splats NULL or not 16-byte aligned", i);
    if (j.keys_capacity < 1 || j.keys_capacity >= ((int64_t)1 << 30))
        return set_error(GS_ERR_INVALID_ARG, "job %d: keys_capacity must be in [1, 2^30)", i);
    if (!j.keys || !j.vals || !j.n_keys || !j.tile_ranges || !j.tile_order)
        return set_error(GS_ERR_INVALID_ARG, "job %d: a key, range or order pointer is NULL", i);
    if (!j.rgb || !j.depth || !j.t_final || !j.last_idx || !j.target_rgb || !j.target_depth || !j.d_rgb ||
        !j.d_depth || !j.loss)
        return set_error(GS_ERR_INVALID_ARG, "job %d: an image, target or loss pointer is NULL", i);
    if (!j.grad2d || ((uintptr_t)j.grad2d & 15))
        return set_error(GS_ERR_INVALID_ARG, "job %d: grad2d NULL or not 16-byte aligned", i);
    if (!j.pose_grad6 || !j.step.pose || !j.step.adam)
        return set_error(GS_ERR_INVALID_ARG, "job %d: pose gradient, pose or Adam state NULL", i);
    if (!(j.step.beta1 >= 0.f && j.step.beta1 < 1.f) || !(j.step.beta2 >= 0.f && j.step.beta2 < 1.f) ||
        !(j.step.eps > 0.f))
        return set_error(GS_ERR_INVALID_ARG, "job %d: bad Adam constants", i);
    if (!j.bwd_workspace || j.bwd_workspace_bytes < gs_project_bwd_ws(j.g.n))
        return set_error(GS_ERR_WORKSPACE, "job %d: backward workspace %zu < %zu bytes", i, j.bwd_workspace_bytes,
                         gs_project_bwd_ws(j.g.n));
    return GS_OK;
}

extern "C" gs_status gs_track_wave(const gs_config* cfg, const gs_track_job* jobs, int32_t n_jobs,
                                   gs_stream stream) {
    if (!cfg) return set_error(GS_ERR_INVALID_ARG, "config is NULL");
    if (!jobs) return set_error(GS_ERR_INVALID_ARG, "jobs is NULL");
    if (n_jobs < 1 || n_jobs > GS_WAVE_MAX)
        return set_error(GS_ERR_INVALID_ARG, "n_jobs %d not in [1, %d]", n_jobs, GS_WAVE_MAX);
    gs_status s;
    WaveBin bins[GS_WAVE_MAX];
    int with_score = 0;
    for (int i = 0; i < n_jobs; ++i) {
        if ((s = job_checks(cfg, jobs[i], i)) != GS_OK) return s;
        if ((s = wave_bin_layout(jobs[i], &bins[i])) != GS_OK) {
            char msg[400];
            snprintf(msg, sizeof(msg), "%s", gs_last_error());
            return set_error(s, "job %d: %s", i, msg);
        }
        with_score += jobs[i].score_terms != nullptr;
    }
    if (with_score != 0 && with_score != n_jobs)
        return set_error(GS_ERR_INVALID_ARG, "score_terms must be given for every job of a wave or for none");
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = wave_project_hist(*cfg, jobs, bins, n_jobs, st)) != GS_OK) return s;
    if ((s = wave_bin_sort(jobs, bins, n_jobs, st)) != GS_OK) return s;
    if ((s = wave_render(*cfg, jobs, n_jobs, st)) != GS_OK) return s;
    return wave_project_bwd(*cfg, jobs, n_jobs, st);
}
