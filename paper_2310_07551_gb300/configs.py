"""Named synthetic workloads (sizes, parameters, step counts, seeds).

Models follow the paper's two test problems (Section 3.1 Schnakenberg,
Section 3.2 FitzHugh-Nagumo) with the parameter sets the workloads fix.
"""
from __future__ import annotations

from dataclasses import dataclass, field


@dataclass(frozen=True)
class Workload:
    name: str
    model: str                 # "schnakenberg" | "fhn"
    dims: tuple[int, ...]      # (n_1, ..., n_d), mode 1 fastest
    lo: float
    hi: float
    tau: float
    steps: int
    params: tuple[float, ...]  # schnakenberg: (gamma, a, b); fhn: (eps, alpha1, alpha0)
    delta: tuple[float, float]
    seed: int = 1

    @property
    def d(self) -> int:
        return len(self.dims)

    @property
    def npoints(self) -> int:
        n = 1
        for v in self.dims:
            n *= v
        return n


SCHNAK = (1000.0, 0.1, 0.9)
FHN = (0.1, 2.0, -0.1)

WORKLOADS: dict[str, Workload] = {
    # 2D Schnakenberg 64^2, FP64, tau = 1e-3, 100 steps
    "schnak2d_64": Workload("schnak2d_64", "schnakenberg", (64, 64), 0.0, 1.0,
                            1e-3, 100, SCHNAK, (1.0, 10.0), seed=1),
    # 2D Schnakenberg 1024^2, tau = 1e-4, 1000 steps
    "schnak2d_1024": Workload("schnak2d_1024", "schnakenberg", (1024, 1024), 0.0, 1.0,
                              1e-4, 1000, SCHNAK, (1.0, 10.0), seed=1),
    # 3D FitzHugh-Nagumo 256^3 on [-1,1]^3, tau = 1e-3, 200 steps
    "fhn3d_256": Workload("fhn3d_256", "fhn", (256, 256, 256), -1.0, 1.0,
                          1e-3, 200, FHN, (1.0, 42.1887), seed=1),
    # 3D FitzHugh-Nagumo 96^3, FP64 forward + adjoint, 200 steps
    "fhn3d_96": Workload("fhn3d_96", "fhn", (96, 96, 96), -1.0, 1.0,
                         1e-3, 200, FHN, (1.0, 42.1887), seed=1),
}
