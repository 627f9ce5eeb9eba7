"""The parity bar of the GPU tests (defined with the oracle, in oracle/parity.py)."""
from oracle.parity import (EDGE_TOL, ID_AGREEMENT, POINT_TOL, T_RTOL, compare,  # noqa: F401
                           edge_distance, hit_points, meets_bar, stats)
