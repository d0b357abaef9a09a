"""The benchmark's algorithmic units (the numerators of its roofline
fractions), checked against hand counts on a two-level hierarchy."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

# finest 10 x 8 x 5 nodes, then a vertical-only coarsening to 3 layers
LEV = [dict(Nx=10, Ny=8, Nz=5, hx=0, hy=0), dict(Nx=10, Ny=8, Nz=3, hx=0, hy=0)]
NODES = 10 * 8 * 5
FREE = 8 * 6 * 4
COLS = 8 * 6


def units(**kw):
    args = dict(levels=LEV, mixed=True, separable=True, solves=[6, 6], nu=(2, 2), cpc=6,
                n_elem=9 * 7 * 4, n_coarse=8 * 6 * 2)
    args.update(kw)
    return {k: dict((b, v) for b, v in u) for k, u in bench.class_units(**args).items()}


def test_separable_smoother_bytes():
    # a group launch reads x of the whole level, f and the factors of its own
    # columns and writes its own x; the first group of each check starts from 0
    u = units()
    g4 = FREE / 4.0
    full = 4 * NODES + 8 * g4 + 144 * COLS / 4.0
    zero = 4 * g4 + 16 * COLS / 4.0 + 4 * NODES
    launches = 12 * 4 * (2 + 2)          # 12 cycles, 4 groups x (2 + 2) sweeps
    checks = 2                            # one per 6 cycles and solve
    assert u["smooth_fine"]["hbm"] == (launches - checks) * full + checks * zero


def test_cold_start_residual_has_no_product():
    # 2 checks plus the warm start's first residual take the row; the cold
    # start reads f and writes the float32 right side and correction only
    u = units()
    assert u["outer_residual"]["fp64"] == 3 * 28.0 * FREE
    assert u["outer_residual"]["hbm"] == 3 * (27 * 8 + 24) * FREE + 16.0 * FREE


def test_float64_transfers_count_their_taps():
    # vertical-only transfer of 5 -> 3 layers: per fine free node one tap
    # (layers kept) or two (layers dropped); per coarse node the centre and
    # the two vertical neighbours, two operations
    u = units(mixed=False, separable=False, cpc=1)
    tz = (5 - 1) + (5 - 3)
    assert u["prolong"]["fp64"] == 12 * float(8 * 6 * tz)
    assert u["restrict"]["fp64"] == 12 * 2.0 * (8 * 6 * 2)


def test_recovery_bytes_of_the_separable_form():
    u = units()
    assert u["recover"] == {"hbm": 2 * ((8 + 24) * NODES + 24.0 * 9 * 7 * 4)}
