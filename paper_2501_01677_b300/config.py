"""One place for the method's constants and run settings.

The paper's own values (Sec. 4.2 w = 0.1; Sec. 4.3 Eq. 11 lambda = 0.41,
lambda_1..4 = 0.05, 0.2, 100, 0.01; Sec. 5.1 30k iterations per group and a 3 x 3
grid of groups), the 3DGS constants it builds on by citation (alpha cutoff and
clamp, termination transmittance, EWA low-pass, Jacobian clamp, near plane,
learning rates, the D-SSIM weight and window), and the settings of this
implementation (tile shape, voting tolerance, autotune cache).  The CUDA library
compiles the rasteriser and loss constants in; `check_library()` verifies that the
values here match the ones it was built with.
"""
from __future__ import annotations

import dataclasses
import json
import os
from typing import Tuple


@dataclasses.dataclass
class PgsagConfig:
    # Sec. 4.2, Eq. 8
    boundary_weight: float = 0.1
    # Sec. 4.3, Eq. 10-11
    lambda_gc: float = 0.41
    lambda_1_mvgeo: float = 0.05
    lambda_2_mvrgb: float = 0.2
    lambda_3_flatten: float = 100.0
    lambda_4_ban: float = 0.01
    # Sec. 5.1
    iterations_per_group: int = 30000
    group_grid: Tuple[int, int] = (3, 3)
    # Sec. 4.1: voting tolerance tau ("empirically selected"; per scene)
    vote_tau: int = 3
    # 3DGS by citation
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    t_min: float = 1e-4
    cov_dilation: float = 0.3
    jac_clamp: float = 1.3
    znear: float = 0.2
    sh_degree: int = 3
    lambda_dssim: float = 0.2
    ssim_window: int = 11
    ssim_sigma: float = 1.5
    learning_rates: Tuple[float, ...] = (1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3)  # means, log-scales, quats, opacity, SH
    adam_betas: Tuple[float, float] = (0.9, 0.999)
    adam_eps: float = 1e-15
    # this implementation
    tile: Tuple[int, int] = (16, 16)
    objective: str = "pg"           # "pg" or "eq11"
    dssim: bool = False
    tsdf_truncation_voxels: float = 4.0
    autotune_cache: str = dataclasses.field(
        default_factory=lambda: os.environ.get("PGSAG_AUTOTUNE_CACHE",
                                               os.path.join(os.path.expanduser("~"), ".cache", "pgsag",
                                                            "autotune.json")))

    def to_json(self) -> str:
        return json.dumps(dataclasses.asdict(self), indent=1, sort_keys=True)

    @staticmethod
    def from_json(text: str) -> "PgsagConfig":
        d = json.loads(text)
        fields = {f.name: f for f in dataclasses.fields(PgsagConfig)}
        out = {}
        for k, v in d.items():
            if k not in fields:
                raise KeyError(f"unknown config key {k}")
            out[k] = tuple(v) if isinstance(v, list) else v
        return PgsagConfig(**out)

    def save(self, path: str) -> None:
        with open(path, "w") as f:
            f.write(self.to_json())

    @staticmethod
    def load(path: str) -> "PgsagConfig":
        with open(path) as f:
            return PgsagConfig.from_json(f.read())

    def check_library(self) -> None:
        """The constants the binding passes or the library compiles in match."""
        from . import _lib as L, raster
        assert abs(L.LAMBDA_GC - self.lambda_gc) < 1e-12
        assert abs(L.LAMBDA_FLAT - self.lambda_3_flatten) < 1e-12
        assert abs(L.LAMBDA_DSSIM - self.lambda_dssim) < 1e-12
        assert abs(raster.LAMBDA_BAN - self.lambda_4_ban) < 1e-12
