"""The learned signed-distance surrogate of one scene: training on exact
distances and use as a broad phase in front of the exact collision test.

Every step runs in the library's kernels (binding.py): exact labels
(vapr_surrogate_samples), training (vapr_mlp_train_step: tcgen05 forward and
backward GEMMs, Adam), inference and the gated collision stage
(vapr_surrogate_collision_cost).  This module only allocates buffers,
shuffles the training set and picks the learning rate of each step.
"""
from __future__ import annotations

import hashlib
import json
import math
import os
import struct

import numpy as np

from . import binding as B
from . import synth

PAD = 0.10     # metres between the cuboids and the edge of the network's domain
MARGIN = 0.05  # spheres within this distance of a surface take the exact test
# Training labels are the exact distance clamped to this band: the gate only
# asks whether a centre is more than r + MARGIN (at most 0.13 m) from every
# surface, so the network need not follow the distance deep inside a cuboid
# or far from all of them.
Y_MIN, Y_MAX = -0.15, 0.40
OVER_WEIGHT = 16.0  # loss weight of overestimates (an overestimate can skip a needed test)


def domain_box(scene: synth.Scene, pad: float = PAD):
    """Axis-aligned box holding every cuboid (corners t + R (+-h)), grown by
    ``pad`` metres."""
    O = scene.n_cuboids
    R = scene.pose[:, :9].reshape(O, 3, 3).astype(np.float64)
    t = scene.pose[:, 9:].astype(np.float64)
    ext = np.einsum("nij,nj->ni", np.abs(R), scene.half_ext.astype(np.float64))
    lo = (t - ext).min(0) - pad
    hi = (t + ext).max(0) + pad
    # float32 box that still contains the float64 one
    lo32 = np.nextafter(lo.astype(np.float32), np.float32(-np.inf))
    hi32 = np.nextafter(hi.astype(np.float32), np.float32(np.inf))
    return lo32, hi32


# ------------------------------------------------------------ checkpoints
# A checkpoint file: the 8-byte magic, a little-endian uint32 header length,
# a JSON header, then the network state's raw bytes as the library keeps
# them (master parameters, Adam moments and step, bfloat16 copies).
CHECKPOINT_MAGIC = b"VAPRMLP1"


def scene_hash(scene: synth.Scene) -> str:
    """SHA-256 of the cuboid poses and half extents (float32 bytes)."""
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(scene.pose, np.float32).tobytes())
    h.update(np.ascontiguousarray(scene.half_ext, np.float32).tobytes())
    return h.hexdigest()


def write_checkpoint(path: str, state: bytes, meta: dict) -> None:
    """Writes meta (JSON) and the raw state bytes; meta gains state_bytes."""
    header = json.dumps({**meta, "state_bytes": len(state)}, sort_keys=True).encode()
    tmp = f"{path}.tmp"
    with open(tmp, "wb") as f:
        f.write(CHECKPOINT_MAGIC)
        f.write(struct.pack("<I", len(header)))
        f.write(header)
        f.write(state)
    os.replace(tmp, path)


def read_checkpoint(path: str) -> tuple[dict, bytes]:
    """(meta, state bytes) of a checkpoint file; ValueError if it is not one
    or is cut short."""
    with open(path, "rb") as f:
        data = f.read()
    if data[:8] != CHECKPOINT_MAGIC or len(data) < 12:
        raise ValueError(f"{path}: not a surrogate checkpoint")
    (hl,) = struct.unpack("<I", data[8:12])
    meta = json.loads(data[12:12 + hl].decode())
    state = data[12 + hl:]
    if len(state) != meta.get("state_bytes"):
        raise ValueError(f"{path}: {len(state)} state bytes, header says {meta.get('state_bytes')}")
    return meta, state


class Surrogate:
    """Network state, domain and training buffers of one scene."""

    def __init__(self, scene: B.DeviceScene, params0, pad: float = PAD, margin: float = MARGIN,
                 device="cuda"):
        import torch
        self.scene = scene
        self.device = device
        self.lo, self.hi = domain_box(scene.host, pad)
        # a hair below pad: room for the float32 rounding of the kernel's
        # outside-the-box distance, which must stay a lower bound
        self.domain = B.surrogate_domain(self.lo, self.hi, pad * (1 - 1e-6), margin)
        self.state = B.alloc_mlp_state(device)
        p0 = torch.as_tensor(np.ascontiguousarray(params0, np.float32), device=device)
        B.vapr_mlp_init(self.state, p0)
        self._ws = {}
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)

    # --------------------------------------------------------------- data
    def samples(self, pts, y_min=-B.FLT_MAX, y_max=B.FLT_MAX):
        """(u, y): domain coordinates and exact distances of points [n, 3]
        (clamped to [y_min, y_max])."""
        import torch
        pts = torch.as_tensor(pts, dtype=torch.float32, device=self.device).contiguous()
        n = pts.shape[0]
        u = torch.empty((n, 3), dtype=torch.float32, device=self.device)
        y = torch.empty(n, dtype=torch.float32, device=self.device)
        B.vapr_surrogate_samples(self.scene, self.domain, pts, n, u, y, y_min, y_max)
        return u, y

    def training_set(self, seed: int, n: int = 2_000_000, near_frac: float = 0.5):
        """Half uniform in the domain box, half near cuboid surfaces; labels
        clamped to [Y_MIN, Y_MAX]."""
        n_near = int(n * near_frac)
        pts = np.concatenate([synth.uniform_points(seed, self.lo, self.hi, n - n_near),
                              synth.near_surface_points(seed, self.scene.host, n_near)])
        return self.samples(pts, Y_MIN, Y_MAX)

    # ----------------------------------------------------------- training
    def workspace(self, batch: int):
        if batch not in self._ws:
            self._ws[batch] = B.alloc_mlp_workspace(batch, self.device)
        return self._ws[batch]

    def train(self, u, y, epochs: int = 80, batch: int = 4096, lr: float = 5e-4,
              lr_final: float = 5e-5, over_weight: float = OVER_WEIGHT, seed: int = 0):
        """Adam over shuffled mini-batches with a cosine learning-rate decay.
        Returns the mean loss of each epoch (read back once per epoch)."""
        import torch
        n = (u.shape[0] // batch) * batch
        steps = epochs * (n // batch)
        ws = self.workspace(batch)
        gen = torch.Generator(device=self.device)
        gen.manual_seed(seed)
        sums = torch.zeros(epochs, dtype=torch.float32, device=self.device)
        k = 0
        for ep in range(epochs):
            perm = torch.randperm(u.shape[0], device=self.device, generator=gen)[:n]
            us, ys = u[perm].contiguous(), y[perm].contiguous()
            for b0 in range(0, n, batch):
                step_lr = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * k / max(steps, 1)))
                B.vapr_mlp_train_step(self.state, us[b0:b0 + batch], ys[b0:b0 + batch], batch,
                                      (step_lr, 0.9, 0.999, 1e-8, over_weight), ws, self.loss)
                sums[ep] += self.loss[0]
                k += 1
        return (sums / (n // batch)).tolist()

    def calibrate(self, seed: int, eta: float, n: int = 200_000):
        """Sets the gate margin from the network's error as judged by the
        exact kernel: on fresh points of the training distribution, the
        largest overestimate delta = max(f - sdf) where sdf lies in the
        training band; margin = max(MARGIN, eta + delta), so that a sphere
        the network clears on such points is at least eta from every
        surface.  Returns delta."""
        n_near = n // 2
        pts = np.concatenate([synth.uniform_points(seed, self.lo, self.hi, n - n_near),
                              synth.near_surface_points(seed, self.scene.host, n_near)])
        u, y = self.samples(pts)
        f = self.forward(u)
        band = (y >= Y_MIN) & (y <= Y_MAX)
        delta = float((f - y)[band].max())
        self.domain.margin = max(MARGIN, eta + delta)
        return delta

    # ---------------------------------------------------------- inference
    def forward(self, u):
        import torch
        u = torch.as_tensor(u, dtype=torch.float32, device=self.device).contiguous()
        out = torch.empty(u.shape[0], dtype=torch.float32, device=self.device)
        B.vapr_mlp_forward(self.state, u, u.shape[0], out)
        return out

    def forward_into(self, u, out):
        B.vapr_mlp_forward(self.state, u, u.shape[0], out)
        return out

    def params(self):
        import torch
        p = torch.empty(B.MLP_PARAMS, dtype=torch.float32, device=self.device)
        B.vapr_mlp_get_params(self.state, p)
        return p

    # -------------------------------------------------------- checkpoints
    def meta(self) -> dict:
        return {"format": 1, "hidden": B.MLP_HIDDEN, "params": B.MLP_PARAMS,
                "scene_sha256": scene_hash(self.scene.host),
                "lo": [float(v) for v in self.lo], "hi": [float(v) for v in self.hi],
                "pad": float(self.domain.pad), "margin": float(self.domain.margin)}

    def save(self, path: str, **extra) -> None:
        """Writes the whole network state (weights, Adam moments and step)
        and the gate domain; `extra` (seed, epochs, ...) goes into the
        header.  The copy to the host waits for the state's pending updates
        on the current stream."""
        write_checkpoint(path, self.state.cpu().numpy().tobytes(), {**extra, **self.meta()})

    def load(self, path: str) -> dict:
        """Restores a state saved by `save` for this scene (same cuboids,
        same library state layout) and its gate margin; training resumes
        where it stopped.  Returns the header."""
        import torch
        meta, state = read_checkpoint(path)
        mine = self.meta()
        for key in ("format", "hidden", "params", "scene_sha256", "lo", "hi", "pad"):
            if meta.get(key) != mine[key]:
                raise ValueError(f"{path}: {key} {meta.get(key)!r} does not match this surrogate's {mine[key]!r}")
        if len(state) != self.state.numel():
            raise ValueError(f"{path}: {len(state)} state bytes, this library keeps {self.state.numel()}")
        host = torch.frombuffer(bytearray(state), dtype=torch.uint8)
        self.state.copy_(host.to(self.state.device))
        self.domain.margin = float(meta["margin"])
        return meta

    def collision_cost(self, robot: B.DeviceRobot, params, pos_packed, n, table, cost=None,
                       dist_packed=None, grad_packed=None, estimate=None, stream=None):
        """vapr_surrogate_collision_cost; returns the estimate tensor [n, S]."""
        import torch
        if estimate is None:
            estimate = torch.empty((n, robot.n_spheres), dtype=torch.float32, device=self.device)
        B.vapr_surrogate_collision_cost(robot, self.scene, params, self.state, self.domain, pos_packed,
                                        n, table, cost, dist_packed, grad_packed, estimate, stream)
        return estimate
