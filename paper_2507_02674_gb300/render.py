"""Frame-level convenience over the binding: upload an environment map and a
G-buffer into device tensors and run the two library calls of a frame
(glint_env_update, glint_shade).  Marshalling only."""
from __future__ import annotations

import numpy as np
import torch

from . import glint
from .synth import EnvMap, GBuffer


def env_tensor(env: EnvMap, device="cuda") -> torch.Tensor:
    t = torch.from_numpy(np.ascontiguousarray(env.texels))
    return t.to(device)


def env_format(env: EnvMap) -> int:
    return glint.FMT_RGBA16F if env.texels.dtype == np.float16 else glint.FMT_RGBA32F


def gbuffer_tensors(gb: GBuffer, device="cuda", pinned: bool = False):
    planes = [torch.from_numpy(np.ascontiguousarray(p.reshape(-1, 4))) for p in gb.planes]
    if device == "cpu":
        return [p.pin_memory() if pinned else p for p in planes]
    return [p.to(device) for p in planes]


def tangent_tensor(gb: GBuffer, device="cuda"):
    return torch.from_numpy(gb.tangents()).to(device)


class Frame:
    """One environment and the buffers to shade G-buffers with it."""

    def __init__(self, ctx: glint.Context, env: EnvMap, cfg: glint.EnvConfig, device="cuda"):
        self.ctx = ctx
        self.cfg = cfg
        self.texels = env_tensor(env, device)
        self.env = glint.Env(ctx, env.width, env.height, env_format(env), env.scale_log2, cfg)

    def update_env(self, stream=None):
        self.env.update(self.texels, stream)

    def shade(self, planes, width: int, height: int, out=None, seed: int = 0, count_mode: int = glint.COUNT_INTEGER,
              debug=None, stream=None, tangent=None, evaluator: int = glint.EVAL_E1, e2_samples: int = 16,
              mlp=None, p_scratch=None, draw: int = glint.DRAW_DUAL, gamma: float = 0.0,
              grid: int = glint.GRID_ISOTROPIC):
        if out is None:
            out = torch.empty(width * height, 4, device=planes[0].device)
        glint.shade(self.ctx, self.env, planes, width, height, out, seed, count_mode, debug, stream, tangent,
                    evaluator, e2_samples, mlp, p_scratch, draw, gamma, grid)
        return out

    def probs(self, planes, width: int, height: int, evaluator: int = glint.EVAL_E1, e2_samples: int = 16,
              tangent=None, mlp=None, out=None, stream=None):
        """p_k of every pixel, (npix, K) on the device."""
        if out is None:
            out = torch.empty(width * height, self.cfg.K, device=planes[0].device)
        glint.reflect_probs(self.ctx, self.env, planes, width, height, out, evaluator, e2_samples, tangent, mlp,
                            stream)
        return out
