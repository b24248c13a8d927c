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


@dataclass(frozen=True)
class Instance:
    dims: tuple[int, int]
    params: tuple[float, float, float]   # (gamma, a, b)
    delta: tuple[float, float]
    tau: float


def batch_instances(count: int = 64, seed: int = 7) -> list[Instance]:
    """Independent Schnakenberg instances with uneven, non-square grids:
    n_1, n_2 from {96, 128, 192, 256, 384, 512}, a in [0.05, 0.2],
    b in [0.7, 1.0], delta_v in [8, 20], tau in [5e-5, 2e-4], gamma = 1000,
    delta_u = 1, domain [0, 1]^2; all drawn from the counter-based generator."""
    from .inputs import uniform01
    sizes = (96, 128, 192, 256, 384, 512)
    r = uniform01(seed, 0, 7 * count).reshape(count, 7)
    out = []
    for k in range(count):
        n1 = sizes[min(int(r[k, 0] * 6), 5)]
        n2 = sizes[min(int(r[k, 1] * 6), 5)]
        a = 0.05 + 0.15 * r[k, 2]
        b = 0.7 + 0.3 * r[k, 3]
        dv = 8.0 + 12.0 * r[k, 4]
        tau = 5e-5 + 1.5e-4 * r[k, 5]
        out.append(Instance((n1, n2), (1000.0, a, b), (1.0, dv), tau))
    return out


BATCH_STEPS = 500
