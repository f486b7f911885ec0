"""One rasterizer iteration over preallocated device buffers.

``Rasterizer`` owns the buffers of one (map size, image grid) pair and chains
the C-ABI calls of include/gs.h: projection -> binning + sort -> forward
compositing -> loss -> backward compositing -> backward projection (+ pose).
Everything runs on the current CUDA stream without host synchronisation, so
an iteration can be captured in a CUDA graph; the key capacity is checked
afterwards through the device status word (``check()``).
"""
from __future__ import annotations

import torch

from . import gs


class Rasterizer:
    def __init__(self, n, cam, cfg=None, rec_dtype=gs.GS_F32, capacity=None, device="cuda"):
        self.n = int(n)
        self.cfg = cfg if cfg is not None else gs.default_config()
        self.rec_dtype = rec_dtype
        self.device = torch.device(device)
        # the pose gradient (6 doubles) and the loss side by side, so that a
        # step's result reads back in one copy (`result`)
        self.result = torch.zeros(7, dtype=torch.float64, device=self.device)
        self.pose = self.result[:6]
        self.set_grid(cam)
        words = gs.SPLAT_WORDS[rec_dtype]
        dt = torch.float32 if rec_dtype == gs.GS_F32 else torch.int32
        self.splats = torch.empty((self.n, words), dtype=dt, device=self.device)
        self.capacity = int(capacity) if capacity is not None else max(4 * self.n, 1024)
        self.keys = torch.empty(max(self.capacity, 1), dtype=torch.int64, device=self.device)
        self.vals = torch.empty(max(self.capacity, 1), dtype=torch.int32, device=self.device)
        self.n_keys = torch.zeros(1, dtype=torch.int64, device=self.device)
        self.grad2d = torch.empty((self.n, gs.GRAD2D_STRIDE), device=self.device)
        self.score = torch.empty((self.n, 2), device=self.device)
        self.loss = torch.zeros(1, dtype=torch.float64, device=self.device)
        self._ws_sort = None
        self._ws_bwd = None
        # the forward records which entries each warp blended and the
        # backward visits only those (same results, fewer visits)
        self.use_blend_masks = True
        self._bm = None

    def set_grid(self, cam):
        """(Re)allocates the image buffers for the camera's sampled grid."""
        Ws, Hs, TX, TY = gs.grid(cam)
        if getattr(self, "_grid", None) == (Ws, Hs, TX, TY):
            return
        self._grid = (Ws, Hs, TX, TY)
        d = self.device
        self.ranges = torch.empty((TX * TY, 2), dtype=torch.int32, device=d)
        self.order = torch.empty(TX * TY, dtype=torch.int32, device=d)
        self.img = {"rgb": torch.empty((3, Hs, Ws), device=d), "depth": torch.empty((Hs, Ws), device=d),
                    "t_final": torch.empty((Hs, Ws), device=d),
                    "last_idx": torch.empty((Hs, Ws), dtype=torch.int32, device=d),
                    "n_blended": torch.empty((Hs, Ws), dtype=torch.int32, device=d)}
        self.dimg = {"d_rgb": torch.empty((3, Hs, Ws), device=d), "d_depth": torch.empty((Hs, Ws), device=d),
                     "loss": self.result[6:7]}
        self._ws_sort = None
        self._ws_pb = None

    def _sort_ws(self, cam_s):
        need = gs.gs_bin_sort_workspace(cam_s, self.rec_dtype, self.n, self.capacity, self.cfg)
        if self._ws_sort is None or self._ws_sort.numel() < need:
            self._ws_sort = gs.workspace(need, self.device)
        return self._ws_sort

    def _pb_ws(self, cam_s, g):
        need = gs.gs_project_bin_sort_workspace(self.cfg, cam_s, g, self.rec_dtype, self.capacity)
        if getattr(self, "_ws_pb", None) is None or self._ws_pb.numel() < need:
            self._ws_pb = gs.workspace(need, self.device)
        return self._ws_pb

    def _project_bin(self, g, cam_s, rebin):
        """Projection, and with rebin the binning + sort fused into it."""
        if rebin:
            gs.gs_project_bin_sort(self.cfg, cam_s, g, self.splats, self.capacity, self.rec_dtype,
                                   ws=self._pb_ws(cam_s, g), keys=self.keys, vals=self.vals, n_keys=self.n_keys,
                                   ranges=self.ranges, order=self.order)
        else:
            gs.gs_project(self.cfg, cam_s, g, self.rec_dtype, self.splats)

    def _masks(self, cam_s):
        if not self.use_blend_masks:
            return None
        need = gs.gs_blend_mask_words(cam_s, self.capacity)
        if self._bm is None or self._bm.numel() < need:
            self._bm = torch.empty(max(need, 1), dtype=torch.int32, device=self.device)
        return self._bm

    def _bwd_ws(self, cam_s, g):
        need = gs.gs_project_bwd_workspace(self.cfg, cam_s, g)
        if self._ws_bwd is None or self._ws_bwd.numel() < need:
            self._ws_bwd = gs.workspace(need, self.device)
        return self._ws_bwd

    # -- stages ------------------------------------------------------------
    def forward(self, g, cam, rebin=True):
        """Projection, binning + sort and forward compositing; returns the
        image buffers (rgb, depth, t_final, last_idx, n_blended).

        rebin=False keeps the tile lists, ranges and order of the last
        binning (the reuse of tile intersection and sorting across the
        iterations of a pruning interval, Sec. 4.1 / Obs. 6): the Gaussians
        are re-projected with the current pose, but each tile composites the
        Gaussians it held when the lists were built."""
        cam_s = cam if isinstance(cam, gs.gs_camera) else gs.camera(cam)
        self.set_grid(cam_s)
        self._project_bin(g, cam_s, rebin)
        self._bm_used = self._masks(cam_s)
        gs.gs_render_fwd(self.cfg, cam_s, self.splats, self.n, self.vals, self.ranges, self.rec_dtype, out=self.img,
                         order=self.order, masks=self._bm_used)
        return self.img

    def loss_grad(self, cam, target_rgb, target_depth):
        cam_s = cam if isinstance(cam, gs.gs_camera) else gs.camera(cam)
        gs.gs_loss_l1(self.cfg, cam_s, self.img["rgb"], self.img["depth"], target_rgb, target_depth, out=self.dimg)
        return self.dimg

    def backward(self, g, cam, d_rgb, d_depth, mode=gs.GS_TRACK, grads=None, want_pose=True, want_score=True):
        cam_s = cam if isinstance(cam, gs.gs_camera) else gs.camera(cam)
        gs.gs_render_bwd(self.cfg, cam_s, g, self.splats, self.vals, self.ranges, self.img["t_final"],
                         self.img["last_idx"], d_rgb, d_depth, mode, self.rec_dtype, grad2d=self.grad2d,
                         grads=grads, pose=self.pose if want_pose else None,
                         score=self.score if want_score else None, ws=self._bwd_ws(cam_s, g), order=self.order,
                         masks=getattr(self, "_bm_used", None))
        return self.grad2d

    def step(self, g, cam, target_rgb, target_depth, mode=gs.GS_TRACK, grads=None, rebin=True):
        """One whole iteration: forward, L1 loss (Eq. 6) and backward."""
        cam_s = cam if isinstance(cam, gs.gs_camera) else gs.camera(cam)
        self.forward(g, cam_s, rebin=rebin)
        self.loss_grad(cam_s, target_rgb, target_depth)
        self.backward(g, cam_s, self.dimg["d_rgb"], self.dimg["d_depth"], mode, grads)
        return self.pose

    def track_step(self, g, cam, target_rgb, target_depth, pose, pose_adam, lr_trans=1e-3, lr_rot=1e-3,
                   rebin=True, wave=True):
        """One fused tracking iteration: projection, binning + sort, forward
        compositing with the loss (gs_render_fwd_loss), backward compositing,
        then backward projection with the pose step fused into its last block
        (gs_project_bwd_step).  `cam` must carry the device pose (`pose`,
        float32 [12]) so the next iteration sees the updated pose; pose_adam
        is the float32 [13] Adam state.  Seven kernel launches: with float32
        records, fresh binning and at most 8192 tiles the iteration runs as a
        wave of one session (gs_track_wave, no memsets) unless wave=False;
        otherwise through the separate calls (the projection also counts the
        binning's tiles, gs_project_bin_sort)."""
        cam_s = cam if isinstance(cam, gs.gs_camera) else gs.camera(cam, pose=pose)
        self.set_grid(cam_s)
        _, _, TX, TY = self._grid
        if wave and rebin and self.rec_dtype == gs.GS_F32 and self.n > 0 and TX * TY <= 8192:
            return self.track_step_wave(g, cam_s, target_rgb, target_depth, pose, pose_adam, lr_trans, lr_rot)
        self._project_bin(g, cam_s, rebin)
        self._bm_used = self._masks(cam_s)
        gs.gs_render_fwd_loss(self.cfg, cam_s, self.splats, self.n, self.vals, self.ranges, target_rgb,
                              target_depth, self.rec_dtype, out=self.img, dimg=self.dimg, order=self.order,
                              masks=self._bm_used)
        gs.gs_render_bwd(self.cfg, cam_s, g, self.splats, self.vals, self.ranges, self.img["t_final"],
                         self.img["last_idx"], self.dimg["d_rgb"], self.dimg["d_depth"], gs.GS_TRACK,
                         self.rec_dtype, grad2d=self.grad2d, order=self.order, masks=self._bm_used)
        gs.gs_project_bwd_step(self.cfg, cam_s, g, self.grad2d, self.pose,
                               gs.pose_step(pose, pose_adam, lr_trans, lr_rot), score=self.score,
                               ws=self._bwd_ws(cam_s, g))
        return self.pose

    def map_step(self, g, cam, target_rgb, target_depth, ms, vs, adam_state, lr=1e-4, rebin=True):
        """One mapping iteration: forward, L1 loss (Eq. 6), backward to the
        2D gradients (GS_MAP), then the backward projection with the map's
        Adam step fused in (gs_project_bwd_adam): g is updated in place, the
        Eq. 7 score terms land in self.score."""
        cam_s = cam if isinstance(cam, gs.gs_camera) else gs.camera(cam)
        self.set_grid(cam_s)
        self._project_bin(g, cam_s, rebin)
        self._bm_used = self._masks(cam_s)
        gs.gs_render_fwd_loss(self.cfg, cam_s, self.splats, self.n, self.vals, self.ranges, target_rgb,
                              target_depth, self.rec_dtype, out=self.img, dimg=self.dimg, order=self.order,
                              masks=self._bm_used)
        gs.gs_render_bwd(self.cfg, cam_s, g, self.splats, self.vals, self.ranges, self.img["t_final"],
                         self.img["last_idx"], self.dimg["d_rgb"], self.dimg["d_depth"], gs.GS_MAP,
                         self.rec_dtype, grad2d=self.grad2d, order=self.order, masks=self._bm_used)
        gs.gs_project_bwd_adam(self.cfg, cam_s, g, self.grad2d, ms, vs, adam_state, lr=lr, score=self.score)

    def track_job(self, g, cam, target_rgb, target_depth, pose, pose_adam, lr_trans=1e-3, lr_rot=1e-3,
                  want_score=True):
        """The descriptor of one track_step of this rasterizer for a wave
        (gs.gs_track_wave): the same buffers, workspaces and pose step.  The
        descriptor holds raw device pointers: g, the targets and this
        rasterizer must outlive every wave that uses it."""
        if self.rec_dtype != gs.GS_F32:
            raise ValueError("waves take float32 records")
        cam_s = cam if isinstance(cam, gs.gs_camera) else gs.camera(cam, pose=pose)
        self.set_grid(cam_s)
        j = gs.gs_track_job()
        j.cam = cam_s
        j.g = gs.gaussians(g)
        j.splats = gs._ptr(self.splats).value
        j.keys_capacity = self.capacity
        pb = self._pb_ws(cam_s, g)
        j.bin_workspace, j.bin_workspace_bytes = gs._ptr(pb).value, pb.numel()
        j.keys, j.vals, j.n_keys = gs._ptr(self.keys).value, gs._ptr(self.vals).value, gs._ptr(self.n_keys).value
        j.tile_ranges, j.tile_order = gs._ptr(self.ranges).value, gs._ptr(self.order).value
        for k in ("rgb", "depth", "t_final", "last_idx", "n_blended"):
            setattr(j, k, gs._ptr(self.img[k]).value)
        bm = self._masks(cam_s)
        self._bm_used = bm
        j.blend_masks = gs._ptr(bm).value if bm is not None else None
        j.target_rgb, j.target_depth = gs._ptr(target_rgb).value, gs._ptr(target_depth).value
        j.d_rgb, j.d_depth = gs._ptr(self.dimg["d_rgb"]).value, gs._ptr(self.dimg["d_depth"]).value
        j.loss = gs._ptr(self.dimg["loss"]).value
        j.grad2d = gs._ptr(self.grad2d).value
        j.pose_grad6 = gs._ptr(self.pose).value
        j.score_terms = gs._ptr(self.score).value if want_score else None
        bw = self._bwd_ws(cam_s, g)
        j.bwd_workspace, j.bwd_workspace_bytes = gs._ptr(bw).value, bw.numel()
        j.step = gs.pose_step(pose, pose_adam, lr_trans, lr_rot)
        return j

    def track_step_wave(self, g, cam, target_rgb, target_depth, pose, pose_adam, lr_trans=1e-3, lr_rot=1e-3):
        """track_step as a wave of one session (gs_track_wave): the same
        iteration in 7 launches, the zeroing the separate calls do with
        memsets (loss, tickets, 2D gradients) folded into the projection
        launch.  The descriptor is rebuilt when a buffer or the camera
        changes."""
        key = (g["means"].data_ptr(), target_rgb.data_ptr(), target_depth.data_ptr(), pose.data_ptr(),
               pose_adam.data_ptr(), float(lr_trans), float(lr_rot),
               bytes(cam) if isinstance(cam, gs.gs_camera) else repr(cam), self.capacity)
        if getattr(self, "_wave_key", None) != key:
            self._wave_job = (gs.gs_track_job * 1)(self.track_job(g, cam, target_rgb, target_depth, pose, pose_adam,
                                                                 lr_trans, lr_rot))
            self._wave_key = key
        gs.gs_track_wave(self.cfg, self._wave_job)
        return self.pose

    def check(self):
        """Synchronises and raises if a device condition was raised (key
        capacity exceeded, a bounded wait that gave up)."""
        code, _ = gs.gs_status_poll(blocking=True)
        if code != gs.GS_OK:
            raise gs.GsError(code, f"device status {code} (n_keys={int(self.n_keys.item())}, "
                                   f"capacity={self.capacity})")


class ListReuse:
    """Tracking with the tile lists reused across a pruning interval (Sec.
    4.1, Obs. 6: the tile-Gaussian intersections barely change from one
    iteration to the next).  The first iteration of an interval bins and
    sorts; the other K - 1 re-project the Gaussians with the current pose and
    composite them through the lists of that binning.  When the interval
    ends, the change ratio of the intersections between the records the
    lists were built from and the records at the current pose decides the
    next interval, gs_next_interval: halved above cfg.change_thr, doubled
    (up to cfg.k_max) below it, starting from cfg.k0.  One host read of the
    ratio per interval."""

    def __init__(self, rast, g):
        self.r = rast
        self.g = g
        self.K = int(rast.cfg.k0)
        self.i = 0
        self.binned = torch.empty_like(rast.splats)  # records the current lists were built from
        self.now = torch.empty_like(rast.splats)
        self.ratio = torch.zeros(1, dtype=torch.float32, device=rast.device)
        self.intervals = []  # (K, change ratio) of every completed interval

    def step(self, cam, target_rgb, target_depth, pose, pose_adam, lr_trans=1e-3, lr_rot=1e-3):
        """One tracking iteration (Rasterizer.track_step); returns whether it
        re-binned."""
        rebin = self.i == 0
        self.r.track_step(self.g, cam, target_rgb, target_depth, pose, pose_adam, lr_trans, lr_rot, rebin=rebin)
        if rebin:
            self.binned.copy_(self.r.splats)
        self.i += 1
        if self.i == self.K:
            cam_s = cam if isinstance(cam, gs.gs_camera) else gs.camera(cam, pose=pose)
            gs.gs_project(self.r.cfg, cam_s, self.g, self.r.rec_dtype, self.now)
            gs.gs_change_ratio(cam_s, self.binned, self.now, self.r.n, self.r.rec_dtype, out=self.ratio,
                               cfg=self.r.cfg)
            r = float(self.ratio.item())
            self.intervals.append((self.K, r))
            self.K = gs.gs_next_interval(self.r.cfg, self.K, r)
            self.i = 0
        return rebin
