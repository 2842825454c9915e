"""The FP32 update forms the MC half slope as
    u = min(|a|, |b|) carrying the sign bit sign(a) xor sign(b)   (PTX min.xorsign.abs)
    h = copysign(max(min(u, |a + b| / 4), 0), a + b)
and claims it equals the definition used everywhere else -- sign(a) min(|a|, |b|,
|a + b| / 4) for a and b of one sign, 0 otherwise (half of van Leer's MC slope) -- up
to the sign of a zero.  Checked here in float32 arithmetic on special values and on
random pairs over many magnitudes, both formulas written out independently."""
import numpy as np


def _xorsign_form(a, b):
    a = a.astype(np.float32)
    b = b.astype(np.float32)
    mag = np.minimum(np.abs(a), np.abs(b)).view(np.uint32)
    sign = (a.view(np.uint32) ^ b.view(np.uint32)) & np.uint32(0x80000000)
    u = (mag | sign).view(np.float32)
    s = (a + b).astype(np.float32)
    q = (np.float32(0.25) * np.abs(s)).astype(np.float32)
    return np.copysign(np.maximum(np.minimum(u, q), np.float32(0.0)), s)


def _definition(a, b):
    a = a.astype(np.float32)
    b = b.astype(np.float32)
    same = ((a > 0) & (b > 0)) | ((a < 0) & (b < 0))
    m = np.minimum(np.minimum(np.abs(a), np.abs(b)),
                   (np.float32(0.25) * np.abs((a + b).astype(np.float32))).astype(np.float32))
    return np.where(same, np.copysign(m, a), np.float32(0.0)).astype(np.float32)


def _check(a, b):
    got, want = _xorsign_form(a, b), _definition(a, b)
    assert np.array_equal(got, want), (a[got != want][:5], b[got != want][:5])


def test_special_values():
    v = np.array([0.0, -0.0, 1.0, -1.0, 3.0, -3.0, 1e-30, -1e-30, 1e30, -1e30,
                  np.float32(1.4e-45), -np.float32(1.4e-45)], dtype=np.float32)
    a, b = np.meshgrid(v, v)
    _check(a.ravel(), b.ravel())


def test_random_pairs_over_magnitudes():
    rng = np.random.default_rng(2208)
    n = 400_000
    mag = np.float32(10.0) ** rng.uniform(-30, 30, size=(2, n)).astype(np.float32)
    sgn = rng.choice(np.array([-1.0, 1.0], dtype=np.float32), size=(2, n))
    a, b = (mag * sgn).astype(np.float32)
    _check(a, b)
    # nearly equal and nearly opposite pairs, where |a + b| / 4 decides
    _check(a, (a * np.float32(1.0001)).astype(np.float32))
    _check(a, (-a * np.float32(0.9999)).astype(np.float32))
