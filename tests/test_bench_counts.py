"""CPU checks of the operation counts behind bench.py's roofline figures.

The roofline fraction of the Cartesian tile kernel divides the implemented
algorithm's operation count by the measured launch time, so the count is
checked here against executed emulations rather than taken on trust:
  * brick_segments equals the number of cell segments that the whole-brick
    line sweeps visit, enumerated tile by tile (ragged last tiles included);
  * eo_product_cost(n, "flop") equals the flops executed by an even-odd 1D
    product that reproduces the plain product A x;
  * eo_segment_costs(n, "flop") equals the flops executed by one segment of
    the z, y and x sweeps (shared even-odd halves, the carried shared node).
"""
import itertools

import numpy as np
import pytest

import bench


class Counter:
    def __init__(self):
        self.flops = 0

    def add(self, a, b):
        self.flops += 1
        return a + b

    def sub(self, a, b):
        self.flops += 1
        return a - b

    def dot(self, row, vec):
        # k multiply-adds = 2k flops
        self.flops += 2 * len(row)
        return float(np.dot(row, vec))


def _halves(cnt, x):
    n = len(x)
    h = n // 2
    e = [cnt.add(x[j], x[n - 1 - j]) for j in range(h)] + ([x[h]] if n % 2 else [])
    o = [cnt.sub(x[j], x[n - 1 - j]) for j in range(h)]
    return e, o


def _blocks(A):
    n = A.shape[0]
    h, ne = n // 2, n - n // 2
    E = np.array([[0.5 * (A[i, j] + A[i, n - 1 - j]) if (j < h and i < h) else A[i, j] for j in range(ne)]
                  for i in range(ne)])
    O = np.array([[0.5 * (A[i, j] - A[i, n - 1 - j]) for j in range(h)] for i in range(h)])
    return E, O


def _apply(cnt, blocks_list, halves_list, n):
    """y = sum over terms of A_t x_t from the even-odd halves (centrosymmetric A_t)."""
    h, ne = n // 2, n - n // 2
    y = np.zeros(n)
    for i in range(h):
        ev = np.concatenate([E[i] for E, _ in blocks_list])
        od = np.concatenate([O[i] for _, O in blocks_list])
        a = cnt.dot(ev, np.concatenate([e for e, _ in halves_list]))
        b = cnt.dot(od, np.concatenate([o for _, o in halves_list]))
        y[i], y[n - 1 - i] = cnt.add(a, b), cnt.sub(a, b)
    if ne > h:
        ev = np.concatenate([E[h] for E, _ in blocks_list])
        y[h] = cnt.dot(ev, np.concatenate([e for e, _ in halves_list]))
    return y


def _centro(rng, n):
    A = rng.standard_normal((n, n))
    return A + A[::-1, ::-1]


@pytest.mark.parametrize("n1", range(2, 10))
def test_eo_product_cost_counts_an_executed_product(n1):
    rng = np.random.default_rng(100 + n1)
    A, x = _centro(rng, n1), rng.standard_normal(n1)
    cnt = Counter()
    halves = _halves(cnt, x)
    y = _apply(cnt, [_blocks(A)], [halves], n1)
    np.testing.assert_allclose(y, A @ x, atol=1e-12)
    assert cnt.flops == bench.eo_product_cost(n1, "flop")


@pytest.mark.parametrize("n1", range(2, 10))
def test_eo_segment_costs_count_executed_segments(n1):
    rng = np.random.default_rng(200 + n1)
    M, K = _centro(rng, n1), _centro(rng, n1)
    x, z = rng.standard_normal(n1), rng.standard_normal(n1)
    carry_a, carry_b = rng.standard_normal(2)
    bm, bk = _blocks(M), _blocks(K)
    costs = []
    # z sweep: ya = M x, yb = K x from one pair of halves, both carried
    cnt = Counter()
    hx = _halves(cnt, x)
    ya, yb = _apply(cnt, [bm], [hx], n1), _apply(cnt, [bk], [hx], n1)
    ya[0], yb[0] = cnt.add(ya[0], carry_a), cnt.add(yb[0], carry_b)
    np.testing.assert_allclose(yb[1:], (K @ x)[1:], atol=1e-12)
    costs.append(cnt.flops)
    # y sweep: ya = M x, yb = K x + M z, both carried
    cnt = Counter()
    hx, hz = _halves(cnt, x), _halves(cnt, z)
    ya, yb = _apply(cnt, [bm], [hx], n1), _apply(cnt, [bk, bm], [hx, hz], n1)
    ya[0], yb[0] = cnt.add(ya[0], carry_a), cnt.add(yb[0], carry_b)
    np.testing.assert_allclose(yb[1:], (K @ x + M @ z)[1:], atol=1e-12)
    costs.append(cnt.flops)
    # x sweep: yb = K x + M z only, carried
    cnt = Counter()
    hx, hz = _halves(cnt, x), _halves(cnt, z)
    yb = _apply(cnt, [bk, bm], [hx, hz], n1)
    yb[0] = cnt.add(yb[0], carry_b)
    costs.append(cnt.flops)
    assert tuple(costs) == bench.eo_segment_costs(n1, "flop")


@pytest.mark.parametrize("degree,cells,tile", [(4, (8, 8, 8), (4, 4, 4)), (4, (9, 7, 5), (4, 4, 4)),
                                               (2, (5, 6, 7), (3, 2, 4)), (5, (3, 3, 3), (3, 3, 3))])
def test_brick_segments_enumerates_the_sweeps(degree, cells, tile):
    seg = [0, 0, 0]
    starts = [range(0, cells[d], tile[d]) for d in range(3)]
    for z0, y0, x0 in itertools.product(starts[2], starts[1], starts[0]):
        nc = [min(tile[0], cells[0] - x0), min(tile[1], cells[1] - y0), min(tile[2], cells[2] - z0)]
        b = [degree * c + 1 for c in nc]
        # every brick line along d, one segment per cell along d
        for d in range(3):
            others = [b[e] for e in range(3) if e != d]
            for _line in range(others[0] * others[1]):
                seg[d] += nc[d]
    assert bench.brick_segments(degree, cells, tile) == (seg[2], seg[1], seg[0])
