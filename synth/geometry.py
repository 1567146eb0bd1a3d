"""TPC readout geometry used by the synthetic events.

36 sectors of 20 degrees (18 per side), 152 pad rows at fixed local x:
63 rows at 0.75 cm pitch from 85.2 cm, 64 rows at 1.0 cm from 135.1 cm and
25 rows at 1.5 cm from 199.4 cm; drift length 250 cm on each side.
Sector k is centred at (k mod 18 + 0.5) * 20 degrees; sectors 0-17 read the
A side (z >= 0) and 18-35 the C side (z < 0).
"""
from dataclasses import dataclass, field
import math
import numpy as np

N_ROWS = 152


def row_radii() -> np.ndarray:
    r = np.arange(N_ROWS, dtype=np.float64)
    x = np.empty(N_ROWS, dtype=np.float64)
    x[:63] = 85.2 + 0.75 * r[:63]
    x[63:127] = 135.1 + 1.0 * (r[63:127] - 63)
    x[127:] = 199.4 + 1.5 * (r[127:] - 127)
    return x


@dataclass
class Geometry:
    n_sectors: int = 36
    row_x: np.ndarray = field(default_factory=row_radii)
    tan_half_sector: float = math.tan(math.radians(10.0))
    z_max: float = 250.0
    alpha0_deg: float = 10.0
    dalpha_deg: float = 20.0

    @property
    def n_rows(self) -> int:
        return int(self.row_x.shape[0])

    def alpha(self, sector: int) -> float:
        return math.radians(self.alpha0_deg + (sector % 18) * self.dalpha_deg)

    @staticmethod
    def side_c(sector: int) -> bool:
        return sector >= 18


def default_geometry() -> Geometry:
    return Geometry()
