"""The hand-written float <-> double conversions of the mixed-precision kernels (IEEE fields
rewritten on the integer pipe, round to nearest with ties to even, hardware conversion only for
zero, subnormal, infinite and NaN results) against IEEE-754 conversion on the host (numpy),
bit for bit: a seeded sweep over the whole float range plus the edge cases where such code goes
wrong (ties, the carry of a rounding into the exponent, FLT_MAX and overflow, the subnormal
boundary, signed zeros, infinities, NaN)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

FLT_MAX = float(np.finfo(np.float32).max)


def _tie_cases():
    """Doubles exactly halfway between two floats (even and odd lower neighbours), just above
    and just below halfway, and ones whose rounding carries into the exponent."""
    rng = np.random.default_rng(21)
    f = rng.standard_normal(4000).astype(np.float32) * np.float32(1e3)
    ex = (f.view(np.uint32) >> 23) & 0xFF
    f = f[(ex > 0) & (ex < 254)]
    fb = f.view(np.uint32).astype(np.uint64)
    d = f.astype(np.float64)
    db = d.view(np.uint64)
    half = np.uint64(1) << np.uint64(28)   # half of one float ulp in the 29 dropped bits
    out = [db + half, db + half + np.uint64(1), db + half - np.uint64(1)]
    # mantissa all ones, then above half: the rounding carries into the exponent
    mant_ones = ((fb[:200] & ~np.uint64(0x7FFFFF)) | np.uint64(0x7FFFFF)).astype(np.uint32).view(np.float32)
    mo = mant_ones.astype(np.float64).view(np.uint64)
    out += [mo + half, mo + half + np.uint64(5)]
    return np.concatenate([o.view(np.float64) for o in out])


def _edge_doubles():
    tiny = float(np.finfo(np.float32).tiny)          # FLT_MIN (smallest normal)
    sub = 2.0 ** -149                                  # smallest subnormal float
    ulp_max = 2.0 ** 104                               # float ulp at FLT_MAX
    vals = [0.0, -0.0, 1.0, -1.0, FLT_MAX, -FLT_MAX, FLT_MAX + ulp_max / 2, FLT_MAX + ulp_max / 2 * (1 - 2 ** -30),
            FLT_MAX * 2, -FLT_MAX * 2, np.inf, -np.inf, np.nan, tiny, -tiny, tiny * (1 - 2 ** -30),
            tiny * (1 + 2 ** -30), tiny / 2, sub, sub / 2, sub / 2 * (1 + 2 ** -20), sub * 1.5, sub * 2.5,
            sub * 0.49, 1e-300, -1e-300, 1e300, 3.0 * 2 ** -127, 2.0 ** -126 - 2.0 ** -150]
    return np.array(vals, dtype=np.float64)


def _sweep_doubles():
    rng = np.random.default_rng(22)
    m = rng.uniform(1.0, 2.0, 200_000)
    e = rng.integers(-160, 135, 200_000)
    s = rng.choice([-1.0, 1.0], 200_000)
    return s * np.ldexp(m, e)


def _check_d2f(pc, d):
    import torch

    with np.errstate(over="ignore"):
        want = d.astype(np.float32)
    got, _ = pc.debug_convert(torch.from_numpy(d), torch.zeros(d.shape[0], dtype=torch.float32))
    got = got.cpu().numpy()
    nan = np.isnan(want)
    assert np.array_equal(np.isnan(got), nan)
    bad = np.nonzero(got[~nan].view(np.uint32) != want[~nan].view(np.uint32))[0]
    assert bad.size == 0, (d[~nan][bad[:5]], got[~nan][bad[:5]], want[~nan][bad[:5]])


def test_double_to_float_sweep(pc):
    _check_d2f(pc, _sweep_doubles())


def test_double_to_float_ties_and_carries(pc):
    _check_d2f(pc, _tie_cases())


def test_double_to_float_edges(pc):
    _check_d2f(pc, _edge_doubles())


def test_float_to_double_is_exact(pc):
    import torch

    rng = np.random.default_rng(23)
    bits = rng.integers(0, 2 ** 32, 300_000, dtype=np.uint64).astype(np.uint32)
    extra = np.array([0, 0x80000000, 1, 0x807FFFFF, 0x00800000, 0x7F7FFFFF, 0x7F800000, 0xFF800000, 0x7FC00000],
                     dtype=np.uint32)
    f = np.concatenate([bits, extra]).view(np.float32)
    _, got = pc.debug_convert(torch.zeros(f.shape[0], dtype=torch.float64), torch.from_numpy(f))
    got = got.cpu().numpy()
    want = f.astype(np.float64)
    nan = np.isnan(want)
    assert np.array_equal(np.isnan(got), nan)
    assert np.array_equal(got[~nan].view(np.uint64), want[~nan].view(np.uint64))
