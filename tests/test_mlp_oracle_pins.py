"""Pins of the learned-kernel network's FP64 oracle: its chain-rule gradient
against central finite differences of its own loss, and GELU / BCE identities."""
import math

import numpy as np

from oracle import mlp_oracle as MO
from paper_1307_3424_gb300 import synth


def small_batch(seed=0, B=6):
    rng = np.random.default_rng(seed)
    x0 = rng.uniform(-1, 1, (B, 3))
    tv = rng.standard_normal((B, MO.N_VAL)) * 0.1
    tm = (rng.uniform(size=(B, MO.N_MASK)) < 0.3).astype(np.float64)
    return x0, tv, tm


def test_gelu_identities():
    z = np.linspace(-4, 4, 17)
    assert MO.gelu(0.0) == 0.0
    assert np.allclose(MO.gelu(z) - MO.gelu(-z), z, atol=1e-15)       # z Phi(z) + z Phi(-z) = z
    h = 1e-6
    assert np.allclose((MO.gelu(z + h) - MO.gelu(z - h)) / (2 * h), MO.gelu_prime(z), atol=1e-8)
    assert abs(MO.gelu_prime(0.0) - 0.5) < 1e-15


def test_bce_at_zero_logit_is_log2():
    y = np.zeros((2, MO.N_OUT))
    tv = np.zeros((2, MO.N_VAL))
    tm = np.full((2, MO.N_MASK), 0.25)
    assert abs(MO.loss(y, tv, tm, 1.0) - math.log(2.0)) < 1e-15


def test_gradient_matches_finite_differences():
    p = synth.mlp_init_params(3).astype(np.float64)
    p[MO.N_PARAMS - MO.N_OUT:] = np.random.default_rng(1).standard_normal(MO.N_OUT) * 0.1   # nonzero b4
    x0, tv, tm = small_batch()
    mw = 0.3
    L0, g = MO.gradients(p, x0, tv, tm, mw)
    assert abs(L0 - MO.loss(MO.forward(p, x0)["y"], tv, tm, mw)) < 1e-15
    rng = np.random.default_rng(2)
    offs, o = [], 0
    for name, shp in MO.SHAPES:      # a few coordinates of every tensor
        n = int(np.prod(shp))
        offs += list(o + rng.choice(n, 4, replace=False))
        o += n
    h = 1e-5
    for i in offs:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (MO.loss(MO.forward(pp, x0)["y"], tv, tm, mw) - MO.loss(MO.forward(pm, x0)["y"], tv, tm, mw)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(g[i])) + 1e-10, (i, fd, g[i])


def test_bf16_rounding():
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 3.14159, -2.5e-3])
    r = MO.round_bf16(v)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2 ** -7     # ties to even
    assert abs(r[3] - 3.140625) < 1e-12 and np.all(np.abs(r - v) <= np.abs(v) * 2 ** -8)
