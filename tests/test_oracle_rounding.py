"""How far the order of FP64 roundings alone moves the oracle, by grid size.

After one step of the benchmark's Terzaghi problem (a strip of columns of it),
the standard and the reassociated builds of the oracle differ by about 3e-14 at
64 rows and by about 1e-12 at 1024 rows: the elliptic solve amplifies FP64
rounding with the grid size.  A relative bar of 1e-12 against the oracle
therefore separates method errors from rounding at small grids only; at large
grids the FP64 GPU path is held to a small multiple of this spread instead
(tests/test_gpu_parity.py).
"""
from rounding_checks import rounding_spread, strip


def test_rounding_order_spread_grows_with_the_grid():
    small, _ = rounding_spread(*strip(64, 16))
    large, _ = rounding_spread(*strip(1024, 128))
    assert small < 2e-13, small
    assert 2e-13 < large < 1e-10, large
    assert large > 5 * small, (small, large)
