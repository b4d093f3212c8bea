"""Pins for the Jacobi oracle: closed forms of the 5-point sweep (CPU only)."""
import numpy as np

from oracle import jacobi as J


def test_constant_field_is_fixed():
    g = np.full((8, 17), 0.75, dtype=np.float32)
    assert np.array_equal(J.run(g, 5), g)


def test_linear_in_columns_is_fixed():
    # f(r, c) = c: (c + c) + ((c - 1) + (c + 1)) = 4c exactly, times 0.25 = c
    g = np.tile(np.arange(33, dtype=np.float32), (12, 1))
    assert np.array_equal(J.step(g), g)


def test_point_source_spreads_to_four_neighbours():
    g = np.zeros((6, 9), dtype=np.float32)
    g[2, 4] = 1.0
    out = J.step(g)
    want = np.zeros_like(g)
    want[1, 4] = want[3, 4] = want[2, 3] = want[2, 5] = 0.25
    assert np.array_equal(out, want)


def test_rows_wrap_around_and_edge_columns_stay():
    g = np.zeros((4, 5), dtype=np.float32)
    g[0, 2] = 4.0
    g[:, 0] = 7.0
    out = J.step(g)
    assert out[3, 2] == 1.0 and out[1, 2] == 1.0          # the ring: row 0's upper neighbour is row 3
    assert np.all(out[:, 0] == 7.0) and np.all(out[:, 4] == 0.0)
    assert out[0, 1] == np.float32((0.0 + 0.0) + (7.0 + 4.0)) * np.float32(0.25)


def test_operation_order_is_fp32():
    # ((a + b) + (c + d)) in fp32 differs from a wider accumulation here
    a, b, c, d = np.float32(1e8), np.float32(-1e8), np.float32(3.0), np.float32(0.5)
    g = np.zeros((3, 3), dtype=np.float32)
    g[0, 1], g[2, 1], g[1, 0], g[1, 2] = a, b, c, d
    out = J.step(g)
    assert out[1, 1] == ((a + b) + (c + d)) * np.float32(0.25)
