"""Lightweight detector descriptions (Sec. 2: barrel layers collapsed at their
average radius, endcap layers at their average z, no modules, a per-layer
material thickness and a uniform solenoid field).

A layer is one of
  * kind 0, barrel cylinder r = pos with z in [lo, hi];
  * kind 1, endcap disk z = pos (signed) with r in [lo, hi].
``x0`` is the thickness in radiation lengths at normal incidence and
``sig_a``/``sig_b`` are the hit resolutions used by the simulation (a: r*phi
direction, b: z on a barrel, r on a disk), all in cm.
"""
from dataclasses import dataclass, field

import numpy as np

KIND_BARREL = 0
KIND_DISK = 1


@dataclass
class Geometry:
    kind: np.ndarray      # int32 [L]
    pos: np.ndarray       # float64 [L]  r (barrel) or signed z (disk), cm
    lo: np.ndarray        # float64 [L]  barrel z_min / disk r_min, cm
    hi: np.ndarray        # float64 [L]  barrel z_max / disk r_max, cm
    x0: np.ndarray        # float64 [L]  x/X0 at normal incidence
    sig_a: np.ndarray     # float64 [L]  r*phi resolution, cm
    sig_b: np.ndarray     # float64 [L]  z (barrel) / r (disk) resolution, cm
    bz: float = 3.8       # tesla
    name: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def n_layers(self) -> int:
        return int(self.kind.shape[0])

    def table(self) -> np.ndarray:
        """[L, 5] float64 rows (kind, pos, lo, hi, x0): the layer table handed to
        both the oracle and the CUDA library."""
        return np.stack([self.kind.astype(np.float64), self.pos, self.lo, self.hi, self.x0], 1)


def _mk(rows, bz, name):
    a = np.array(rows, dtype=np.float64)
    return Geometry(kind=a[:, 0].astype(np.int32), pos=a[:, 1].copy(), lo=a[:, 2].copy(),
                    hi=a[:, 3].copy(), x0=a[:, 4].copy(), sig_a=a[:, 5].copy(),
                    sig_b=a[:, 6].copy(), bz=bz, name=name)


def geometry_barrel10(sigma=0.01, x0=0.01, bz=3.8):
    """Idealised barrel: 10 cylinders r = 4..100 cm evenly spaced, |z| < 100 cm."""
    rows = [(KIND_BARREL, 4.0 + 96.0 * i / 9.0, -100.0, 100.0, x0, sigma, sigma) for i in range(10)]
    return _mk(rows, bz, "barrel10")


def geometry_barrel14(sigma=0.01, x0=0.01, bz=3.8):
    """The same idealised barrel with 14 evenly spaced cylinders r = 4..100 cm
    (used for the fixed-assignment fit with 14 hits per track)."""
    rows = [(KIND_BARREL, 4.0 + 96.0 * i / 13.0, -100.0, 100.0, x0, sigma, sigma) for i in range(14)]
    return _mk(rows, bz, "barrel14")


def geometry_cmslike(bz=3.8):
    """CMS-like tracker stand-in: 4 pixel barrels (r = 3, 7, 11, 16 cm, |z| < 27),
    10 strip barrels (r = 25..110 cm, |z| < 110), 3 pixel disks per side
    (|z| = 30, 40, 50 cm, r in [4.5, 16]) and 9 strip disks per side
    (|z| = 120..280 cm, r in [22, 110]); 38 surfaces.  Material rises linearly
    from 0.01 X0 (innermost) to 0.04 X0 (outermost) with the layer index inside
    the barrel and inside each endcap.  Resolutions: pixel 0.002 cm in both
    directions, strip 0.003 cm (r*phi) x 1 cm (z or r)."""
    rows = []
    pix_r = [3.0, 7.0, 11.0, 16.0]
    strip_r = [25.0 + 85.0 * i / 9.0 for i in range(10)]
    for i, r in enumerate(pix_r + strip_r):
        x0 = 0.01 + 0.03 * i / 13.0
        if i < 4:
            rows.append((KIND_BARREL, r, -27.0, 27.0, x0, 0.002, 0.002))
        else:
            rows.append((KIND_BARREL, r, -110.0, 110.0, x0, 0.003, 1.0))
    disk_z = [30.0, 40.0, 50.0] + [120.0 + 160.0 * i / 8.0 for i in range(9)]
    for side in (+1.0, -1.0):
        for j, z in enumerate(disk_z):
            x0 = 0.01 + 0.03 * j / 11.0
            if j < 3:
                rows.append((KIND_DISK, side * z, 4.5, 16.0, x0, 0.002, 0.002))
            else:
                rows.append((KIND_DISK, side * z, 22.0, 110.0, x0, 0.003, 1.0))
    return _mk(rows, bz, "cmslike38")
