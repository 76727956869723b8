"""Frame-to-frame odometry with HGMM registration.

Each frame's GMM tree (hgmm_build) is the model the next frame is registered
to (hgmm_register); the relative motions are concatenated into sensor poses
(the paper chains its frame-to-frame VLP-16 registrations into a trajectory,
Sec. 6).  The previous motion seeds each registration (constant-velocity
start); because the descent of Algorithm 1 is local, a turn that the
previous motion does not predict can land it in a wrong basin, so each frame
is also registered from that start yawed by a few degrees about the sensor's
vertical axis and the result with the lowest Eq. 11 objective is kept (the
choice is made on the device: no host round trip per frame).  Two trees
alternate: while frame k is registered to the tree of frame k-1 on one
stream, the tree of frame k is built on another; CUDA events order a build
after the registration that last used its tree and a registration after the
build of its model.
"""
from __future__ import annotations

import numpy as np

from . import binding as B


def _torch():
    import torch
    return torch


def yaw(deg: float) -> np.ndarray:
    """4x4 rotation by `deg` degrees about the z (vertical) axis."""
    a = np.radians(deg)
    T = np.eye(4)
    T[:2, :2] = [[np.cos(a), -np.sin(a)], [np.sin(a), np.cos(a)]]
    return T


class Odometry:
    """`yaw_starts_deg`: the yaw offsets of the starts tried per frame (the
    first should be 0, the constant-velocity start itself)."""

    def __init__(self, max_points: int, depth: int = 4, iters: int = 30, overlap: bool = True,
                 prm: B.hgmm_params | None = None, yaw_starts_deg=(0.0, 3.0, -3.0)):
        torch = _torch()
        self.depth, self.iters, self.prm = depth, iters, prm
        self.trees = [B.Tree(max_points, depth), B.Tree(max_points, depth)]
        self.overlap = overlap
        self.s_reg = torch.cuda.Stream()
        self.s_build = torch.cuda.Stream() if overlap else self.s_reg
        self.yaws = [float(d) for d in yaw_starts_deg]
        if not self.yaws:
            raise ValueError("yaw_starts_deg: at least one start")
        self.Rz = torch.from_numpy(np.stack([yaw(d).reshape(16) for d in self.yaws])).cuda()
        self.T0 = torch.zeros(16, dtype=torch.float64, device="cuda")
        self.Tc = torch.zeros(16, dtype=torch.float64, device="cuda")
        self.obj = torch.zeros(2, dtype=torch.float64, device="cuda")  # [best, candidate]

    def run(self, frames):
        """Relative motions (F, 4, 4) on the device for a list of F frames
        ((N, 4) float32 CUDA tensors): T_rel[k] maps frame k into frame k-1,
        T_rel[0] = I.  All work is enqueued on the object's streams; the
        returned tensor is ready once `sync()` returns."""
        torch = _torch()
        F = len(frames)
        T = torch.zeros((F, 16), dtype=torch.float64, device="cuda")
        T[0, [0, 5, 10, 15]] = 1.0
        built = [torch.cuda.Event() for _ in range(F)]
        used = [torch.cuda.Event() for _ in range(F)]
        # the motion tensor is written by the registration stream
        self.s_reg.wait_stream(torch.cuda.current_stream())
        self.s_build.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(self.s_build):
            self.trees[0].build(frames[0], self.depth, self.prm, stream=self.s_build)
            built[0].record(self.s_build)
        for k in range(1, F):
            model, nxt = self.trees[(k - 1) % 2], self.trees[k % 2]
            with torch.cuda.stream(self.s_reg):
                self.s_reg.wait_event(built[k - 1])
                self._register(model, frames[k], T[k - 1], T[k])
                used[k].record(self.s_reg)
            if k + 1 < F:
                with torch.cuda.stream(self.s_build):
                    if k >= 2:
                        self.s_build.wait_event(used[k - 1])  # tree k % 2 was the model of frame k - 1
                    nxt.build(frames[k], self.depth, self.prm, stream=self.s_build)
                    built[k].record(self.s_build)
        return T.view(F, 4, 4)

    def _register(self, model, src, T_prev, T_out):
        """Registration of `src` to `model` from each start Rz(yaw) T_prev;
        T_out receives the result with the lowest objective (ties keep the
        earlier start).  Enqueued on the registration stream."""
        for s, d in enumerate(self.yaws):
            if d == 0.0:
                T0 = T_prev
            else:
                B.hgmm_pose_compose(self.Rz[s:s + 1], T_prev.view(1, 16), self.T0.view(1, 16), stream=self.s_reg)
                T0 = self.T0
            dst, o = (T_out, self.obj[0:1]) if s == 0 else (self.Tc, self.obj[1:2])
            model.register(src, T_init=T0, iters=self.iters, stream=self.s_reg, T_out=dst)
            B.hgmm_register_objective(model.handle, o, stream=self.s_reg)
            if s > 0:
                B.hgmm_pose_select(T_out.view(1, 16), self.obj[0:1], self.Tc.view(1, 16), self.obj[1:2],
                                   T_out.view(1, 16), stream=self.s_reg, obj_out=self.obj[0:1])

    def sync(self):
        for t in self.trees:
            t.sync(self.s_reg)
            t.sync(self.s_build)


def chain(T_rel):
    """Sensor poses W[k] = W[k-1] T_rel[k] (W[0] = I) of host motions (F, 4, 4)."""
    T_rel = np.asarray(T_rel, np.float64)
    W = np.empty_like(T_rel)
    W[0] = np.eye(4)
    for k in range(1, T_rel.shape[0]):
        W[k] = W[k - 1] @ T_rel[k]
    return W
