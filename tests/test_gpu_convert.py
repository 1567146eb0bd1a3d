"""The float <-> double conversions of the mixed-precision kernels
(widen / narrow, rebuilt on the integer pipes instead of the FP64-pipe
conversion instructions), compared bit by bit with the IEEE conversions.

widen is exact for zero, normal, infinite and NaN floats and maps float
subnormals to zero.  narrow rounds to nearest with ties away from zero (IEEE:
ties to even), flushes results below float's normal range, saturates beyond
float's range (to within 8 ulp of the largest float) and turns infinities and NaNs into NaN.  Off those cases the two
must agree bit for bit."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _run(f=None, d=None):
    import torch
    import paper_2502_09138_gb300 as G
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda() if a is not None else None
    w, n = G.diag_convert(t(f), t(d))
    torch.cuda.synchronize()
    return (w.cpu().numpy() if w is not None else None), (n.cpu().numpy() if n is not None else None)


def test_widen_bitwise():
    rng = np.random.default_rng(11)
    bits = rng.integers(0, 2 ** 32, 1 << 20, dtype=np.uint64).astype(np.uint32)
    special = np.array([0.0, -0.0, 1.0, -1.0, np.inf, -np.inf, np.finfo(np.float32).max,
                        np.finfo(np.float32).tiny, -np.finfo(np.float32).tiny], np.float32).view(np.uint32)
    f = np.concatenate([bits, special]).view(np.float32)
    w, _ = _run(f=f)
    ref = f.astype(np.float64)
    sub = (np.abs(f) < np.finfo(np.float32).tiny) & (f != 0)
    nan = np.isnan(f)
    ok = ~sub & ~nan
    assert np.array_equal(w[ok].view(np.uint64), ref[ok].view(np.uint64))
    assert np.all(w[sub] == 0.0)
    assert np.all(np.isnan(w[nan]))


def test_narrow_bitwise_and_ties():
    rng = np.random.default_rng(12)
    # doubles across float's normal range (random mantissas: no ties)
    e = rng.integers(-120, 120, 1 << 20)
    d = rng.uniform(1.0, 2.0, 1 << 20) * np.exp2(e.astype(np.float64)) * rng.choice([-1.0, 1.0], 1 << 20)
    _, n = _run(d=d)
    ref = d.astype(np.float32)
    assert np.array_equal(n.view(np.uint32), ref.view(np.uint32))
    # exact ties: the midpoint of two adjacent floats rounds away from zero
    base = rng.uniform(1.0, 2.0, 4096).astype(np.float32) * np.float32(2.0) ** rng.integers(-100, 100, 4096)
    up = np.nextafter(base, np.float32(np.inf))
    mid = (base.astype(np.float64) + up.astype(np.float64)) / 2
    for sign in (1.0, -1.0):
        _, n = _run(d=sign * mid)
        assert np.array_equal(n, (sign * up).astype(np.float32))
    # beyond float's range: a finite float within 8 ulp of the largest (the
    # exponent saturates, the fraction keeps its top bits); infinities, NaN: NaN
    _, n = _run(d=np.array([1e300, -1e300, np.inf, np.nan]))
    b = n.view(np.uint32)
    assert 0x7F7FFFF8 <= b[0] <= 0x7F7FFFFF and 0xFF7FFFF8 <= b[1] <= 0xFF7FFFFF
    assert np.isnan(n[2]) and np.isnan(n[3])
