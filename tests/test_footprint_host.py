"""Host check of the staging-tile bound of the tiled restriction and nested-source
kernels: the source rows a block of consecutive targets spans, decided on the exact
fixed-point positions of the interface (the oracle's model of them), never exceed
ceil((targets - 1) b) + ORD + 2 (b = target spacing / source spacing), the footprint the
launcher sizes the tiles with: the stencil starts of a block lie at most
ceil((targets - 1) b) apart, plus the stencil's ORD + 1 rows, plus one row of slack for
the fixed-point rounding of b (a bound two rows short fails here).  No GPU."""
import math

import numpy as np

from oracle import interp


def _starts(T, n_src, order):
    one = 1 << interp.FIX_BITS
    if order == 1:
        return [min(max(int(t) >> interp.FIX_BITS, 0), n_src - 2) for t in T]
    half = one >> 1
    return [min(max((int(t) + half) >> interp.FIX_BITS, 1), n_src - 2) - 1 for t in T]


def test_block_footprint_bounds_the_staged_rows():
    rng = np.random.default_rng(11)
    for _ in range(400):
        order = int(rng.integers(1, 3))
        targets = int(rng.choice([16, 64]))
        lim = {16: 20, 64: 80}[targets]
        # spacing ratios the tiled form admits: (targets - 1) b + order + 2 <= lim
        b = float(rng.uniform(0.05, (lim - order - 2) / (targets - 1)))
        h_src = 1e-4
        n_src = 400
        n_dst = int(rng.integers(targets, 4 * targets))
        a = float(rng.uniform(0.0, n_src - 2 - (n_dst - 1) * b))  # nested: every target inside
        T = interp._fixed_positions(0.0, h_src, a * h_src, b * h_src, n_dst)
        starts = _starts(T, n_src, order)
        bound = math.ceil((targets - 1) * b) + order + 2
        assert bound <= lim
        for b0 in range(0, n_dst, targets):
            blk = [starts[min(b0 + i, n_dst - 1)] for i in range(targets)]  # past the end: the last target
            span = blk[-1] - blk[0] + order + 1
            assert span <= bound, (order, targets, b, a, b0, span, bound)
